// Batched execution of the many tiny contractions near the leaves of a tree.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

constexpr int MICRO_D = 12;          // dimensions per operand group
constexpr int64_t MICRO_MAX = 4096;  // entries (all items) of every tensor of a micro node
constexpr int MICRO_NODES = 64;      // nodes per micro subtree
constexpr int MICRO_BETA = 1024;     // batch items a micro kernel handles

// One tiny pairwise contraction, all offsets relative to the program arena
// (elements) and to the maxima / argmax buffers.
struct MicroDesc {
    int32_t nout, nk, pow2, nbeta;
    int32_t nout_total, ktotal;
    int64_t offA, offB, offC;
    int32_t bsa, bsb;
    int32_t osz[MICRO_D], osh[MICRO_D], osa[MICRO_D], osb[MICRO_D];
    int32_t ksz[MICRO_D], ksh[MICRO_D], ksa[MICRO_D], ksb[MICRO_D];
    int64_t mxa, mxb, mxc;           // maximum slots (-1: none)
    int32_t mxa_bs, mxb_bs;
    int64_t amoff;                   // argmax offset (-1: none)
};

template <typename T>
void launch_micro(const MicroDesc *nodes, const int32_t *sub_beg, int nsub, int semiring, T *arena,
                  unsigned long long *mx, int32_t *am, cudaStream_t st);

}  // namespace tn

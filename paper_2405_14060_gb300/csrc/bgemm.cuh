// Batched strided GEMM over label groups (CUDA cores, sum-product).
//
// A pairwise contraction C = sum_K A (x) B (Def. "Tensor Network" for two
// tensors) whose labels split into
//   G: in A, B and C (a batch of independent products),
//   M: in A and C only,   N: in B and C only,   K: in A and B only (summed),
// is the batched matrix product C[g, m, n] = sum_k A[g, m, k] B[g, k, n],
// whatever the order of the labels in each operand.  Each (tensor, group)
// pair gets a table of the flat offsets of every index of the group (the sum
// of digit x stride over the group's labels), so an element's address is the
// sum of three table entries and the operands are read where they lie: no
// permutation pass in HBM.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

struct BDesc {
    int64_t G, M, N, K;            // group sizes per batch item
    int nbeta;                     // batch items (evidence sets) of C
    int64_t bsa, bsb, bsc;         // per-item strides (0: the operand lacks the batch label)
    // offset tables (device, int32, one buffer): A by g, B by g, C by g,
    // A by m, C by m, B by n, C by n, A by k, B by k
    const int32_t *tag, *tbg, *tcg, *tam, *tcm, *tbn, *tcn, *tak, *tbk;
    int a_kfast;                   // A's fastest label is summed (else it is in M or G)
    int b_kfast;                   // B's fastest label is summed (else in N or G)
    int c_nfast;                   // C's fastest label is in N (else in M or G)
    int c_gfast;                   // a G label lies inside C's 32-byte sectors: tiles
                                   // enumerate G fastest, so that the tiles writing
                                   // the same sectors run together (their partial
                                   // writes merge in L2 instead of each eviction
                                   // costing a DRAM read-modify-write)
    const void *A, *B;
    void *C;
    const unsigned long long *mxa, *mxb;
    int mxa_bs, mxb_bs;            // 1 if the maximum is per item, else 0
    unsigned long long *mxc;       // per-item maximum of C
    int nsplit;                    // K split over this many blocks (partials in scratch)
    int64_t kchunk;                // summed indices per split (a multiple of the K tile)
    int tile;                      // tile shape id (see bgemm.cu); -1: does not fit
    int tc;                        // 1: tensor-core gather kernel (float data, no K split)
    int *err;                      // set by a bounded device wait that gave up (tc kernel)
};

// Scratch bytes of the split-K partials (0 when the K space is not split).
size_t bgemm_scratch_bytes(const BDesc &d, int elem_bytes);
// Choose the tile shape and the K split of a descriptor (host); sets tile to
// -1 when the contraction exceeds the kernels' index ranges.
void bgemm_configure(BDesc &d, int elem_bytes);
template <typename T>
void launch_bgemm(const BDesc &d, void *scratch, cudaStream_t st);
int bgemm_launches(const BDesc &d);
// The tensor-core form (tcgather.cu): tiles of 128 rows, and its launch.
int64_t tc_gather_tiles(const BDesc &d);
void launch_tc_gather(const BDesc &d, cudaStream_t st);

}  // namespace tn

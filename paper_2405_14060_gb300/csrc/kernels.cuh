// Device-side descriptors shared by the executor and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

constexpr int MAXD = 32;     // dimensions of a contraction after fusion

// One pairwise contraction C = (+)_K A (x) B over strided operands.
//   output dims (C's storage order, row-major, batch outermost):
//     osz[d], stride in A osa[d], stride in B osb[d] (0 = operand lacks it)
//   summed dims (flat K index row-major over them): ksz, ksa, ksb
//   batch: nbeta items; operand batch strides bsa / bsb (0 = no batch label)
// Scaling (sum-product): each operand has a per-item maximum (double bits,
// mxa / mxb, indexed by item * mxa_bs); the kernel multiplies A by
// 2^-e(A) and B by 2^-e(B) before the product, where e(.) is the binary
// exponent of the maximum, and records the maximum of C in mxc.
struct CDesc {
    int nout, nk;
    int nbeta;
    int pow2;                 // every size is a power of two
    int64_t nout_total;       // per batch item
    int64_t ktotal;
    int32_t osz[MAXD], osh[MAXD];
    int64_t osa[MAXD], osb[MAXD];
    int32_t ksz[MAXD], ksh[MAXD];
    int64_t ksa[MAXD], ksb[MAXD];
    int64_t bsa, bsb;
    const void *A, *B;
    void *C;
    const unsigned long long *mxa, *mxb;
    int mxa_bs, mxb_bs;       // 1 if the maximum is per item, else 0
    unsigned long long *mxc;  // per item maximum of C (NULL: not recorded)
    int32_t *argmax;          // max-plus: flat K index of the maximiser
};

enum Semiring { SUM = 0, MAXPLUS = 1 };

template <typename T>
void launch_contract(const CDesc &d, int semiring, void *scratch, size_t scratch_bytes,
                     cudaStream_t st, int *nlaunch);
size_t contract_scratch_bytes(const CDesc &d, int elem_bytes);
bool contract_uses_splitk(const CDesc &d);
template <typename T>
bool launch_contract_splitk_fixed(const CDesc &d, int semiring, void *scratch, size_t cap,
                                  cudaStream_t st);

}  // namespace tn

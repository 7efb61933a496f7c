// Micro-subtree kernel: one CTA evaluates, node after node, every pairwise
// contraction of one small subtree of the contraction tree (forward), or the
// adjoint contractions of its nodes in reverse order (backward), with a
// block-wide barrier between nodes.  Subtrees are independent, so one launch
// covers all of them; this replaces thousands of launches of microsecond-size
// kernels near the leaves of a tree (factor tensors absorbing unity vectors,
// fields and couplings) by one.
#include <cmath>

#include "devutil.cuh"
#include "kernels.cuh"
#include "micro.cuh"

namespace tn {

template <typename T, int SEMI>
__global__ void __launch_bounds__(256) k_micro(const MicroDesc *__restrict__ nodes,
                                               const int32_t *__restrict__ sub_beg, T *arena,
                                               unsigned long long *mx, int32_t *am) {
    __shared__ unsigned long long smx[MICRO_BETA];
    const int i0 = sub_beg[blockIdx.x], i1 = sub_beg[blockIdx.x + 1];
    for (int i = i0; i < i1; ++i) {
        const MicroDesc &d = nodes[i];
        const int nb = d.nbeta, nout = d.nout_total;
        T tmax = 0;   // single item: this thread's maximum, reduced once per node
        for (int b = threadIdx.x; b < nb; b += blockDim.x) smx[b] = 0ull;
        __syncthreads();
        for (int idx = threadIdx.x; idx < nb * nout; idx += blockDim.x) {
            int beta = idx / nout, o = idx - beta * nout;
            int64_t oa = d.offA + (int64_t)beta * d.bsa, ob = d.offB + (int64_t)beta * d.bsb;
            if (d.pow2) {
                for (int q = 0; q < d.nout; ++q) {
                    int dg = (o >> d.osh[q]) & (d.osz[q] - 1);
                    oa += dg * d.osa[q];
                    ob += dg * d.osb[q];
                }
            } else {
                int r = o;
                for (int q = d.nout - 1; q >= 0; --q) {
                    int dg = r % d.osz[q];
                    r /= d.osz[q];
                    oa += dg * d.osa[q];
                    ob += dg * d.osb[q];
                }
            }
            const T *A = arena + oa;
            const T *B = arena + ob;
            if (SEMI == SUM) {
                T sa = d.mxa >= 0 ? pow2neg<T>(exp_of_bits(mx[d.mxa + beta * d.mxa_bs])) : T(1);
                T sb = d.mxb >= 0 ? pow2neg<T>(exp_of_bits(mx[d.mxb + beta * d.mxb_bs])) : T(1);
                T acc = 0;
                for (int k = 0; k < d.ktotal; ++k) {
                    int ka = 0, kb = 0;
                    if (d.pow2) {
                        for (int q = 0; q < d.nk; ++q) {
                            int dg = (k >> d.ksh[q]) & (d.ksz[q] - 1);
                            ka += dg * d.ksa[q];
                            kb += dg * d.ksb[q];
                        }
                    } else {
                        int r = k;
                        for (int q = d.nk - 1; q >= 0; --q) {
                            int dg = r % d.ksz[q];
                            r /= d.ksz[q];
                            ka += dg * d.ksa[q];
                            kb += dg * d.ksb[q];
                        }
                    }
                    acc += A[ka] * B[kb];
                }
                acc *= sa * sb;   // exact: both are powers of two
                arena[d.offC + idx] = acc;
                if (d.mxc >= 0) {
                    if (nb == 1) tmax = tmax > acc ? tmax : acc;
                    else if (acc > T(0)) atomicMax(&smx[beta], dbits((double)acc));
                }
            } else {
                // operands max-normalised by their recorded maxima
                const T oa_ = d.mxa >= 0 ? okey_off<T>(mx[d.mxa + beta * d.mxa_bs]) : T(0);
                const T ob_ = d.mxb >= 0 ? okey_off<T>(mx[d.mxb + beta * d.mxb_bs]) : T(0);
                T best = -INFINITY;
                int32_t bk = 0;
                for (int k = 0; k < d.ktotal; ++k) {
                    int ka = 0, kb = 0, r = k;
                    for (int q = d.nk - 1; q >= 0; --q) {
                        int dg = r % d.ksz[q];
                        r /= d.ksz[q];
                        ka += dg * d.ksa[q];
                        kb += dg * d.ksb[q];
                    }
                    T v = (A[ka] - oa_) + (B[kb] - ob_);
                    if (v > best) { best = v; bk = k; }
                }
                arena[d.offC + idx] = best;
                if (d.amoff >= 0) am[d.amoff + idx] = bk;
                if (d.mxc >= 0 && isfinite((double)best)) atomicMax(&smx[beta], okey((double)best));
            }
        }
        if (SEMI == SUM && d.mxc >= 0 && nb == 1) {
            // one shared atomic per warp instead of one per output
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                T v = __shfl_xor_sync(0xffffffffu, tmax, o);
                tmax = tmax > v ? tmax : v;
            }
            if ((threadIdx.x & 31) == 0 && tmax > T(0)) atomicMax(&smx[0], dbits((double)tmax));
        }
        __syncthreads();
        if (d.mxc >= 0)
            for (int b = threadIdx.x; b < nb; b += blockDim.x) mx[d.mxc + b] = smx[b];
        __syncthreads();
    }
}

template <typename T>
void launch_micro(const MicroDesc *nodes, const int32_t *sub_beg, int nsub, int semiring, T *arena,
                  unsigned long long *mx, int32_t *am, cudaStream_t st) {
    if (nsub <= 0) return;
    if (semiring == SUM) k_micro<T, SUM><<<nsub, 256, 0, st>>>(nodes, sub_beg, arena, mx, am);
    else k_micro<T, MAXPLUS><<<nsub, 256, 0, st>>>(nodes, sub_beg, arena, mx, am);
}

template void launch_micro<float>(const MicroDesc *, const int32_t *, int, int, float *,
                                  unsigned long long *, int32_t *, cudaStream_t);
template void launch_micro<double>(const MicroDesc *, const int32_t *, int, int, double *,
                                   unsigned long long *, int32_t *, cudaStream_t);

}  // namespace tn

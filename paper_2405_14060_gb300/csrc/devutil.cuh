// Small device helpers shared by the kernels: binary exponents of recorded
// maxima, exact power-of-two scale factors, per-item maximum recording.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tn {

__device__ __forceinline__ int exp_of_bits(unsigned long long b) {
    if (b == 0ull) return 0;
    return (int)((b >> 52) & 0x7ffull) - 1023;
}

template <typename T> __device__ __forceinline__ T pow2neg(int e);
template <> __device__ __forceinline__ float pow2neg<float>(int e) {
    e = max(-126, min(126, e));
    return __int_as_float((127 - e) << 23);
}
template <> __device__ __forceinline__ double pow2neg<double>(int e) {
    e = max(-1022, min(1022, e));
    return __longlong_as_double((long long)(1023 - e) << 52);
}

// Asynchronous global -> shared copies (one element per call) and their
// commit / wait groups; a thread that only reads the shared slots it copied
// itself needs no barrier, only the wait.
__device__ __forceinline__ void cp_async_el(float *smem, const float *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_el(double *smem, const double *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Quotient and remainder of a non-negative tile index by a positive count:
// a shift when the count is a power of two (lb = its log2, else -1), 32-bit
// division when both fit, 64-bit division otherwise.
__device__ __forceinline__ int64_t div_tile(int64_t a, int64_t b, int lb, int64_t &rem) {
    int64_t q;
    if (lb >= 0) q = a >> lb;
    else if (((uint64_t)a | (uint64_t)b) < (1ull << 32)) q = (int64_t)((uint32_t)a / (uint32_t)b);
    else q = a / b;
    rem = a - q * b;
    return q;
}
__host__ __device__ __forceinline__ int log2_if_pow2(int64_t b) {
    if (b <= 0 || (b & (b - 1))) return -1;
    int l = 0;
    while ((1ll << l) < b) ++l;
    return l;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}

// Record per-item maxima of non-negative values: one atomic per warp when the
// warp's lanes share an item, else one per lane.  Every lane of the warp must
// call it.
__device__ __forceinline__ void record_max(unsigned long long *mx, int64_t beta, bool active,
                                           double v) {
    if (!mx) return;
    unsigned long long m = active ? dbits(v) : 0ull;
    long long b0 = __shfl_sync(0xffffffffu, (long long)beta, 0);
    bool same = __all_sync(0xffffffffu, !active || beta == b0);
    if (same) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, m, s);
            m = o > m ? o : m;
        }
        if ((threadIdx.x & 31) == 0 && m) atomicMax(mx + b0, m);
    } else if (active && m) {
        atomicMax(mx + beta, m);
    }
}

// Block-wide maximum of non-negative values, one atomic per block.  Every
// thread of the block must call it (it synchronises the block).
__device__ __forceinline__ void block_max_atomic(unsigned long long *mx, double v) {
    __shared__ unsigned long long sm[32];
    unsigned long long m = dbits(v > 0 ? v : 0.0);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, m, s);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t = sm[w] > t ? sm[w] : t;
        if (mx && t) atomicMax(mx, t);
    }
}

// Max-plus offsets (max-normalisation of tropical tensors): a tensor's
// maximum is recorded under an order-preserving 64-bit key, so that
// atomicMax orders signed values; key 0 sorts below every double and means
// "not recorded".  A consumer subtracts the recorded maximum of each operand
// before adding them, so stored tropical tensors stay near zero and FP32
// rounding acts on small magnitudes; the offsets are summed in FP64.
__device__ __forceinline__ unsigned long long okey(double d) {
    unsigned long long b = (unsigned long long)__double_as_longlong(d);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
// The offset of a recorded key: 0 when nothing, or a non-finite maximum (an
// all -inf tensor), was recorded.
template <typename T>
__device__ __forceinline__ T okey_off(unsigned long long k) {
    if (k == 0ull) return T(0);
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d = __longlong_as_double((long long)b);
    return isfinite(d) ? (T)d : T(0);
}
// Record the maxima of signed values: one atomic per warp when the warp's
// lanes share an item, else one per lane.  Every lane of the warp calls it.
__device__ __forceinline__ void record_max_key(unsigned long long *mx, int64_t beta, bool active,
                                               double v) {
    if (!mx) return;
    double m = active ? v : -INFINITY;
    long long b0 = __shfl_sync(0xffffffffu, (long long)beta, 0);
    bool same = __all_sync(0xffffffffu, !active || beta == b0);
    if (same) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((threadIdx.x & 31) == 0 && isfinite(m)) atomicMax(mx + b0, okey(m));
    } else if (active && isfinite(m)) {
        atomicMax(mx + beta, okey(m));
    }
}

// Grid shape for an item-parallel kernel: blockIdx.y is the batch item and
// blockIdx.x strides over the item's entries; about 16 blocks per SM overall.
inline dim3 item_grid(int64_t per_item, int nbeta, int threads = 256) {
    int64_t want = (per_item + threads - 1) / threads;
    int64_t cap = (152LL * 16) / (nbeta > 0 ? nbeta : 1);
    if (cap < 1) cap = 1;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return dim3((unsigned)want, (unsigned)(nbeta > 0 ? nbeta : 1), 1);
}

}  // namespace tn

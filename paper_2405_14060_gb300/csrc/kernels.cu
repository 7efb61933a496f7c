// Generic pairwise-contraction kernels (sm_103a, CUDA cores).
//
// One pairwise contraction C_{Vc} = (+)_{(Va u Vb) \ Vc} A_{Va} (x) B_{Vb}
// (Def. "Tensor Network" restricted to two tensors; Eq. tropical for the
// max-plus semiring) over operands with arbitrary label strides, so that no
// operand has to be permuted in HBM first.
//
//   k_contract        one thread per output entry, loop over the summed
//                     space; coalesced when consecutive outputs map to
//                     consecutive entries of the streamed operand.
//   k_contract_splitk the summed space split over blocks (small outputs:
//                     root traces, adjoints of small factors); partial results
//                     reduced in a fixed order by k_splitk_reduce, so results
//                     are deterministic.
//
// Sum-product rescaling: each operand is multiplied by 2^-e, e the binary
// exponent of its recorded maximum, before the product (exact in binary
// floating point), and the kernel records the maximum of its output, so every
// stored tensor stays near 1 whatever the model's scale.  The exponents are
// summed into log Z by k_logz.
#include <cfloat>
#include <cmath>

#include "devutil.cuh"
#include "kernels.cuh"

namespace tn {

// offsets of output entry o in A and B
__device__ __forceinline__ void decode_out(const CDesc &d, int64_t o, int64_t &oa, int64_t &ob) {
    if (d.pow2) {
#pragma unroll 4
        for (int i = 0; i < d.nout; ++i) {
            int64_t dig = (o >> d.osh[i]) & (int64_t)(d.osz[i] - 1);
            oa += dig * d.osa[i];
            ob += dig * d.osb[i];
        }
    } else {
        for (int i = d.nout - 1; i >= 0; --i) {
            int64_t dig = o % d.osz[i];
            o /= d.osz[i];
            oa += dig * d.osa[i];
            ob += dig * d.osb[i];
        }
    }
}

__device__ __forceinline__ void decode_k(const CDesc &d, int64_t k, int64_t &ka, int64_t &kb) {
    ka = 0;
    kb = 0;
    if (d.pow2) {
#pragma unroll 4
        for (int i = 0; i < d.nk; ++i) {
            int64_t dig = (k >> d.ksh[i]) & (int64_t)(d.ksz[i] - 1);
            ka += dig * d.ksa[i];
            kb += dig * d.ksb[i];
        }
    } else {
        for (int i = d.nk - 1; i >= 0; --i) {
            int64_t dig = k % d.ksz[i];
            k /= d.ksz[i];
            ka += dig * d.ksa[i];
            kb += dig * d.ksb[i];
        }
    }
}

template <typename T, int SEMI>
__global__ void __launch_bounds__(256) k_contract(const __grid_constant__ CDesc d) {
    const int64_t beta = blockIdx.y;
    T mx = 0;
    T sa = T(1), sb = T(1);
    // max-plus: operands max-normalised by their recorded maxima
    T oa_ = T(0), ob_ = T(0), mxq = -INFINITY;
    if (SEMI == SUM) {
        sa = d.mxa ? pow2neg<T>(exp_of_bits(d.mxa[beta * d.mxa_bs])) : T(1);
        sb = d.mxb ? pow2neg<T>(exp_of_bits(d.mxb[beta * d.mxb_bs])) : T(1);
    } else {
        oa_ = d.mxa ? okey_off<T>(d.mxa[beta * d.mxa_bs]) : T(0);
        ob_ = d.mxb ? okey_off<T>(d.mxb[beta * d.mxb_bs]) : T(0);
    }
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < d.nout_total;
         o += (int64_t)gridDim.x * blockDim.x) {
        int64_t oa = beta * d.bsa, ob = beta * d.bsb;
        decode_out(d, o, oa, ob);
        const T *A = (const T *)d.A + oa;
        const T *B = (const T *)d.B + ob;
        const int64_t idx = beta * d.nout_total + o;
        if (SEMI == SUM) {
            T acc = 0;
            if (d.nk == 0) {
                acc = (A[0] * sa) * (B[0] * sb);
            } else if (d.nk == 1) {
                int64_t sA = d.ksa[0], sB = d.ksb[0];
#pragma unroll 4
                for (int64_t k = 0; k < d.ktotal; ++k) acc += (A[k * sA] * sa) * (B[k * sB] * sb);
            } else {
                for (int64_t k = 0; k < d.ktotal; ++k) {
                    int64_t ka, kb;
                    decode_k(d, k, ka, kb);
                    acc += (A[ka] * sa) * (B[kb] * sb);
                }
            }
            ((T *)d.C)[idx] = acc;
            mx = mx > acc ? mx : acc;
        } else {
            T best = -INFINITY;
            int32_t bk = 0;
            if (d.nk == 0) {
                best = (A[0] - oa_) + (B[0] - ob_);
            } else if (d.nk == 1) {
                int64_t sA = d.ksa[0], sB = d.ksb[0];
                for (int64_t k = 0; k < d.ktotal; ++k) {
                    T v = (A[k * sA] - oa_) + (B[k * sB] - ob_);
                    if (v > best) { best = v; bk = (int32_t)k; }
                }
            } else {
                for (int64_t k = 0; k < d.ktotal; ++k) {
                    int64_t ka, kb;
                    decode_k(d, k, ka, kb);
                    T v = (A[ka] - oa_) + (B[kb] - ob_);
                    if (v > best) { best = v; bk = (int32_t)k; }
                }
            }
            ((T *)d.C)[idx] = best;
            if (d.argmax) d.argmax[idx] = bk;
            mxq = mxq > best ? mxq : best;
        }
    }
    if (SEMI == SUM && d.mxc) block_max_atomic(d.mxc + beta, (double)mx);
    if (SEMI == MAXPLUS) record_max_key(d.mxc, beta, true, (double)mxq);
}

// ---------------------------------------------------------------- split-K

template <typename T, int SEMI>
__global__ void __launch_bounds__(256) k_contract_splitk(const __grid_constant__ CDesc d,
                                                         int64_t chunk, int nchunks, T *part,
                                                         int32_t *pidx) {
    int64_t oy = (int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (oy >= d.nout_total * d.nbeta) return;
    int64_t beta = oy / d.nout_total, o = oy - beta * d.nout_total;
    int64_t oa = beta * d.bsa, ob = beta * d.bsb;
    decode_out(d, o, oa, ob);
    const T *A = (const T *)d.A + oa;
    const T *B = (const T *)d.B + ob;
    int64_t k0 = (int64_t)blockIdx.x * chunk;
    int64_t k1 = min(k0 + chunk, d.ktotal);
    __shared__ T sv[32];
    __shared__ int32_t si[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (SEMI == SUM) {
        T sa = d.mxa ? pow2neg<T>(exp_of_bits(d.mxa[beta * d.mxa_bs])) : T(1);
        T sb = d.mxb ? pow2neg<T>(exp_of_bits(d.mxb[beta * d.mxb_bs])) : T(1);
        T acc = 0;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            int64_t ka, kb;
            decode_k(d, k, ka, kb);
            acc += (A[ka] * sa) * (B[kb] * sb);
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
        if (lane == 0) sv[wid] = acc;
        __syncthreads();
        if (wid == 0) {
            T v = lane < (int)(blockDim.x >> 5) ? sv[lane] : T(0);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
            if (lane == 0) part[oy * nchunks + blockIdx.x] = v;
        }
    } else {
        const T oa_ = d.mxa ? okey_off<T>(d.mxa[beta * d.mxa_bs]) : T(0);
        const T ob_ = d.mxb ? okey_off<T>(d.mxb[beta * d.mxb_bs]) : T(0);
        T best = -INFINITY;
        int32_t bk = INT32_MAX;
        for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            int64_t ka, kb;
            decode_k(d, k, ka, kb);
            T s = (A[ka] - oa_) + (B[kb] - ob_);
            if (s > best || (s == best && (int32_t)k < bk)) { best = s; bk = (int32_t)k; }
        }
        // (max, lowest index) reduction
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            T ov = __shfl_xor_sync(0xffffffffu, best, s);
            int32_t oi = __shfl_xor_sync(0xffffffffu, bk, s);
            if (ov > best || (ov == best && oi < bk)) { best = ov; bk = oi; }
        }
        if (lane == 0) { sv[wid] = best; si[wid] = bk; }
        __syncthreads();
        if (wid == 0) {
            bool ok = lane < (int)(blockDim.x >> 5);
            T v = ok ? sv[lane] : T(-INFINITY);
            int32_t i = ok ? si[lane] : INT32_MAX;
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                T ov = __shfl_xor_sync(0xffffffffu, v, s);
                int32_t oi = __shfl_xor_sync(0xffffffffu, i, s);
                if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
            }
            if (lane == 0) {
                part[oy * nchunks + blockIdx.x] = v;
                pidx[oy * nchunks + blockIdx.x] = i;
            }
        }
    }
}

template <typename T, int SEMI>
__global__ void __launch_bounds__(256) k_splitk_reduce(const __grid_constant__ CDesc d,
                                                       int nchunks, const T *part,
                                                       const int32_t *pidx) {
    int64_t oy = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t total = d.nout_total * d.nbeta;
    bool active = oy < total;
    int64_t beta = active ? oy / d.nout_total : 0;
    T val = 0;
    if (active) {
        if (SEMI == SUM) {
            T acc = 0;
            for (int c = 0; c < nchunks; ++c) acc += part[oy * nchunks + c];
            val = acc;
        } else {
            // chunks in increasing K order: a strictly larger value replaces
            // the incumbent, so ties keep the lowest index
            T best = part[oy * nchunks];
            int32_t bi = pidx[oy * nchunks];
            for (int c = 1; c < nchunks; ++c) {
                T v = part[oy * nchunks + c];
                if (v > best) { best = v; bi = pidx[oy * nchunks + c]; }
            }
            if (bi == INT32_MAX) bi = 0;
            val = best;
            if (d.argmax) d.argmax[oy] = bi;
        }
        ((T *)d.C)[oy] = val;
    }
    if (SEMI == SUM) record_max(d.mxc, beta, active, (double)val);
    else record_max_key(d.mxc, beta, active, (double)val);
}

static constexpr int64_t kTargetThreads = 152LL * 2048;

static void splitk_shape(const CDesc &d, int64_t &chunk, int &nchunks) {
    int64_t outs = d.nout_total * d.nbeta;
    int64_t want_blocks = std::max<int64_t>(1, kTargetThreads / 256 / std::max<int64_t>(1, outs));
    chunk = std::max<int64_t>(1024, (d.ktotal + want_blocks - 1) / want_blocks);
    nchunks = (int)((d.ktotal + chunk - 1) / chunk);
}

// Split the summed space over blocks when the outputs alone cannot fill the
// GPU and each output sums enough terms to make the serial loop the bottleneck.
static bool use_splitk(const CDesc &d) {
    int64_t outs = d.nout_total * d.nbeta;
    return d.ktotal >= 256 && outs * 64 < kTargetThreads * 4 && outs <= (1LL << 20);
}

bool contract_uses_splitk(const CDesc &d) { return use_splitk(d); }

size_t contract_scratch_bytes(const CDesc &d, int elem_bytes) {
    if (!use_splitk(d)) return 0;
    int64_t chunk;
    int nchunks;
    splitk_shape(d, chunk, nchunks);
    int64_t n = d.nout_total * d.nbeta * nchunks;
    size_t b = (size_t)n * elem_bytes;
    b = (b + 255) & ~(size_t)255;
    return b + (size_t)n * 4;
}

template <typename T>
void launch_contract(const CDesc &d, int semiring, void *scratch, size_t scratch_bytes,
                     cudaStream_t st, int *nlaunch) {
    int64_t total = d.nout_total * d.nbeta;
    if (total == 0) return;
    if (use_splitk(d) && scratch && scratch_bytes >= contract_scratch_bytes(d, sizeof(T))) {
        int64_t chunk;
        int nchunks;
        splitk_shape(d, chunk, nchunks);
        int64_t n = total * nchunks;
        size_t pb = ((size_t)n * sizeof(T) + 255) & ~(size_t)255;
        T *part = (T *)scratch;
        int32_t *pidx = (int32_t *)((char *)scratch + pb);
        dim3 grid((unsigned)nchunks, (unsigned)std::min<int64_t>(total, 65535),
                  (unsigned)((total + 65534) / 65535));
        if (semiring == SUM)
            k_contract_splitk<T, SUM><<<grid, 256, 0, st>>>(d, chunk, nchunks, part, pidx);
        else
            k_contract_splitk<T, MAXPLUS><<<grid, 256, 0, st>>>(d, chunk, nchunks, part, pidx);
        unsigned rb = (unsigned)((total + 255) / 256);
        if (semiring == SUM)
            k_splitk_reduce<T, SUM><<<rb, 256, 0, st>>>(d, nchunks, part, pidx);
        else
            k_splitk_reduce<T, MAXPLUS><<<rb, 256, 0, st>>>(d, nchunks, part, pidx);
        if (nlaunch) *nlaunch += 2;
        return;
    }
    dim3 grid = item_grid(d.nout_total, d.nbeta);
    if (semiring == SUM)
        k_contract<T, SUM><<<grid, 256, 0, st>>>(d);
    else
        k_contract<T, MAXPLUS><<<grid, 256, 0, st>>>(d);
    if (nlaunch) *nlaunch += 1;
}

// Contraction with any scratch in a fixed buffer of `cap` bytes: outputs
// whose summed space is long enough for split-K (the choice launch_contract
// makes) keep their partial results there, the others run on k_contract,
// which needs no scratch.  The K-chunk count of split-K is bounded so that
// outputs x chunks stay near kTargetThreads / 256, hence its partials hold at
// most a few thousand entries.  Returns false (launching nothing) when the
// output has more than cap / (element size + 4) entries, the limit stated for
// callers whatever the path.
template <typename T>
bool launch_contract_splitk_fixed(const CDesc &d, int semiring, void *scratch, size_t cap,
                                  cudaStream_t st) {
    int64_t total = d.nout_total * d.nbeta;
    if (total == 0) return true;
    if ((size_t)total * (sizeof(T) + 4) > cap) return false;
    if (!use_splitk(d)) {
        launch_contract<T>(d, semiring, nullptr, 0, st, nullptr);
        return true;
    }
    int64_t chunk;
    int nchunks;
    splitk_shape(d, chunk, nchunks);
    size_t pb = ((size_t)(total * nchunks) * sizeof(T) + 255) & ~(size_t)255;
    if (pb + (size_t)(total * nchunks) * 4 > cap) return false;
    T *part = (T *)scratch;
    int32_t *pidx = (int32_t *)((char *)scratch + pb);
    dim3 grid((unsigned)nchunks, (unsigned)std::min<int64_t>(total, 65535),
              (unsigned)((total + 65534) / 65535));
    if (semiring == SUM)
        k_contract_splitk<T, SUM><<<grid, 256, 0, st>>>(d, chunk, nchunks, part, pidx);
    else
        k_contract_splitk<T, MAXPLUS><<<grid, 256, 0, st>>>(d, chunk, nchunks, part, pidx);
    unsigned rb = (unsigned)((total + 255) / 256);
    if (semiring == SUM) k_splitk_reduce<T, SUM><<<rb, 256, 0, st>>>(d, nchunks, part, pidx);
    else k_splitk_reduce<T, MAXPLUS><<<rb, 256, 0, st>>>(d, nchunks, part, pidx);
    return true;
}

template bool launch_contract_splitk_fixed<float>(const CDesc &, int, void *, size_t, cudaStream_t);
template bool launch_contract_splitk_fixed<double>(const CDesc &, int, void *, size_t,
                                                   cudaStream_t);

template void launch_contract<float>(const CDesc &, int, void *, size_t, cudaStream_t, int *);
template void launch_contract<double>(const CDesc &, int, void *, size_t, cudaStream_t, int *);

}  // namespace tn

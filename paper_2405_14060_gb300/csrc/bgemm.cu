// Batched strided GEMM kernels (CUDA cores): contractions whose row, column
// or summed group is too small for the tensor-core tiles and whose operands
// are both too large to stream against a small one (bgemm.cuh).
//
//   k_bgemm      one block per (item, g, m tile, n tile, K split); the A and B
//                tiles are gathered through the offset tables into shared
//                memory (double-buffered, the next tile's loads in flight
//                during the current tile's multiply-adds), each thread keeps a
//                TM x TN register tile whose rows and columns are strided by
//                the thread grid, so that consecutive lanes store consecutive
//                entries along C's fastest group.
//   k_bgemm_fin  when K is split: sums the split partials in split order
//                (deterministic), applies the operands' power-of-two scales,
//                stores C and records its per-item maximum.
//
// Sum-product rescaling as in every other kernel: A and B enter multiplied by
// 2^-e (e the binary exponent of their recorded maxima; applied to the
// accumulated product, which is exact in binary floating point) and the
// kernel records the maximum of C.
#include <algorithm>
#include <cmath>

#include "bgemm.cuh"
#include "devutil.cuh"

namespace tn {

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 16;

template <typename T, int BM, int BN, int TM, int TN, bool NFAST>
__global__ void __launch_bounds__(kThreads) k_bgemm(const __grid_constant__ BDesc d, T *part) {
    constexpr int MT = BM / TM, NT = BN / TN;
    static_assert(MT * NT == kThreads, "thread grid");
    constexpr int LA = BM * kBK / kThreads, LB = BN * kBK / kThreads;
    static_assert(LA >= 1 && LB >= 1, "tile loads");
    __shared__ T As[2][kBK][BM + 1];
    __shared__ T Bs[2][kBK][BN + 1];
    const int tid = threadIdx.x;
    // block -> (m tile, n tile, g, item, split), m tiles fastest
    int64_t b = blockIdx.x;
    const int64_t tiles_m = (d.M + BM - 1) / BM, tiles_n = (d.N + BN - 1) / BN;
    const int64_t tmi = b % tiles_m;
    b /= tiles_m;
    const int64_t tni = b % tiles_n;
    b /= tiles_n;
    const int64_t g = b % d.G;
    b /= d.G;
    const int64_t beta = b % d.nbeta;
    const int split = (int)(b / d.nbeta);
    const int64_t m0 = tmi * BM, n0 = tni * BN;
    const int64_t kbeg = (int64_t)split * d.kchunk;
    const int64_t kend = min(d.K, kbeg + d.kchunk);
    const T *Ab = (const T *)d.A + beta * d.bsa + d.tag[g];
    const T *Bb = (const T *)d.B + beta * d.bsb + d.tbg[g];
    // fixed parts of this thread's tile loads: the m (n) offsets when the
    // operand is read along its m (n) group, else the k index
    int32_t aoff[LA], boff[LB];
    int ak[LA], bk[LB];
#pragma unroll
    for (int r = 0; r < LA; ++r) {
        const int e = tid + kThreads * r;
        const int m = d.a_kfast ? e / kBK : e % BM;
        ak[r] = d.a_kfast ? e % kBK : e / BM;
        aoff[r] = m0 + m < d.M ? __ldg(d.tam + m0 + m) : -1;
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
        const int e = tid + kThreads * r;
        const int n = d.b_kfast ? e / kBK : e % BN;
        bk[r] = d.b_kfast ? e % kBK : e / BN;
        boff[r] = n0 + n < d.N ? __ldg(d.tbn + n0 + n) : -1;
    }
    T ra[LA], rb[LB];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int64_t k = k0 + ak[r];
            ra[r] = (aoff[r] >= 0 && k < kend) ? Ab[aoff[r] + __ldg(d.tak + k)] : T(0);
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int64_t k = k0 + bk[r];
            rb[r] = (boff[r] >= 0 && k < kend) ? Bb[boff[r] + __ldg(d.tbk + k)] : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int e = tid + kThreads * r;
            const int m = d.a_kfast ? e / kBK : e % BM;
            As[buf][ak[r]][m] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int e = tid + kThreads * r;
            const int n = d.b_kfast ? e / kBK : e % BN;
            Bs[buf][bk[r]][n] = rb[r];
        }
    };
    const int im = NFAST ? tid / NT : tid % MT;
    const int in = NFAST ? tid % NT : tid / MT;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    int buf = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
        __syncthreads();
        for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
            const bool more = k0 + kBK < kend;
            if (more) load(k0 + kBK);
#pragma unroll
            for (int kk = 0; kk < kBK; ++kk) {
                T a[TM], bv[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][im + i * MT];
#pragma unroll
                for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][in + j * NT];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * bv[j];
            }
            if (more) {
                store(buf ^ 1);
                __syncthreads();
                buf ^= 1;
            }
        }
    }
    if (d.nsplit > 1) {
        // unscaled partials, dense [split][item][g][n][m]
        T *P = part + (((int64_t)split * d.nbeta + beta) * d.G + g) * d.M * d.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t m = m0 + im + i * MT;
            if (m >= d.M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int64_t n = n0 + in + j * NT;
                if (n < d.N) P[n * d.M + m] = acc[i][j];
            }
        }
        return;
    }
    T sa = d.mxa ? pow2neg<T>(exp_of_bits(d.mxa[beta * d.mxa_bs])) : T(1);
    T sb = d.mxb ? pow2neg<T>(exp_of_bits(d.mxb[beta * d.mxb_bs])) : T(1);
    const T s = sa * sb;
    T *Cb = (T *)d.C + beta * d.bsc + d.tcg[g];
    T mx = 0;
    int32_t cn[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int64_t n = n0 + in + j * NT;
        cn[j] = n < d.N ? __ldg(d.tcn + n) : -1;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t m = m0 + im + i * MT;
        if (m >= d.M) continue;
        const int32_t cm = __ldg(d.tcm + m);
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            if (cn[j] < 0) continue;
            const T v = acc[i][j] * s;
            Cb[cm + cn[j]] = v;
            mx = mx > v ? mx : v;
        }
    }
    if (d.mxc) block_max_atomic(d.mxc + beta, (double)mx);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_bgemm_fin(const __grid_constant__ BDesc d,
                                                        const T *part) {
    const int64_t per = d.G * d.M * d.N, total = per * d.nbeta;
    const int64_t o = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = o < total;
    int64_t beta = 0;
    T v = 0;
    if (active) {
        beta = o / per;
        int64_t r = o - beta * per;
        const int64_t g = r / (d.M * d.N);
        r -= g * d.M * d.N;
        const int64_t n = r / d.M, m = r - n * d.M;
        T acc = 0;
        for (int sp = 0; sp < d.nsplit; ++sp) acc += part[(int64_t)sp * total + o];
        T sa = d.mxa ? pow2neg<T>(exp_of_bits(d.mxa[beta * d.mxa_bs])) : T(1);
        T sb = d.mxb ? pow2neg<T>(exp_of_bits(d.mxb[beta * d.mxb_bs])) : T(1);
        v = acc * (sa * sb);
        ((T *)d.C)[beta * d.bsc + d.tcg[g] + d.tcm[m] + d.tcn[n]] = v;
    }
    record_max(d.mxc, beta, active, (double)v);
}

// tile shapes: 0 = wide (n > 16), 1 = narrow (n <= 16)
template <typename T>
struct Tiles;
template <>
struct Tiles<float> {
    static constexpr int BM0 = 128, BN0 = 64, TM0 = 8, TN0 = 4;
    static constexpr int BM1 = 256, BN1 = 16, TM1 = 8, TN1 = 2;
};
template <>
struct Tiles<double> {
    static constexpr int BM0 = 64, BN0 = 64, TM0 = 4, TN0 = 4;
    static constexpr int BM1 = 128, BN1 = 16, TM1 = 4, TN1 = 2;
};

void tile_dims(const BDesc &d, int esz, int &bm, int &bn) {
    if (esz == 8) {
        bm = d.tile ? Tiles<double>::BM1 : Tiles<double>::BM0;
        bn = d.tile ? Tiles<double>::BN1 : Tiles<double>::BN0;
    } else {
        bm = d.tile ? Tiles<float>::BM1 : Tiles<float>::BM0;
        bn = d.tile ? Tiles<float>::BN1 : Tiles<float>::BN0;
    }
}

}  // namespace

void bgemm_configure(BDesc &d, int elem_bytes) {
    d.tile = d.N <= 16 ? 1 : 0;
    int bm, bn;
    tile_dims(d, elem_bytes, bm, bn);
    const int64_t blocks = ((d.M + bm - 1) / bm) * ((d.N + bn - 1) / bn) * d.G * d.nbeta;
    // split the summed space when the output tiles alone leave most SMs idle
    // and every split still runs several K tiles; partials stay under 1 GiB
    int64_t ns = 1;
    const int64_t want = 152LL * 3;
    if (blocks < want && d.K >= 8 * kBK) {
        ns = std::min<int64_t>((want + blocks - 1) / blocks, d.K / (4 * kBK));
        const int64_t outs = d.G * d.M * d.N * d.nbeta;
        while (ns > 1 && (double)ns * outs * elem_bytes > (double)(1LL << 30)) ns /= 2;
        ns = std::max<int64_t>(1, ns);
    }
    int64_t chunk = (d.K + ns - 1) / ns;
    chunk = (chunk + kBK - 1) / kBK * kBK;
    d.kchunk = std::max<int64_t>(chunk, kBK);
    d.nsplit = (int)((d.K + d.kchunk - 1) / d.kchunk);
    if (d.nsplit < 1) d.nsplit = 1;
}

size_t bgemm_scratch_bytes(const BDesc &d, int elem_bytes) {
    if (d.nsplit <= 1) return 0;
    return (size_t)d.nsplit * (size_t)(d.G * d.M * d.N * d.nbeta) * (size_t)elem_bytes;
}

int bgemm_launches(const BDesc &d) { return d.nsplit > 1 ? 2 : 1; }

template <typename T>
void launch_bgemm(const BDesc &d, void *scratch, cudaStream_t st) {
    const int64_t outs = d.G * d.M * d.N * d.nbeta;
    if (outs == 0) return;
    int bm, bn;
    tile_dims(d, (int)sizeof(T), bm, bn);
    const int64_t blocks =
        ((d.M + bm - 1) / bm) * ((d.N + bn - 1) / bn) * d.G * d.nbeta * d.nsplit;
    T *part = (T *)scratch;
    using Ti = Tiles<T>;
    if (d.tile == 0) {
        if (d.c_nfast)
            k_bgemm<T, Ti::BM0, Ti::BN0, Ti::TM0, Ti::TN0, true>
                <<<(unsigned)blocks, kThreads, 0, st>>>(d, part);
        else
            k_bgemm<T, Ti::BM0, Ti::BN0, Ti::TM0, Ti::TN0, false>
                <<<(unsigned)blocks, kThreads, 0, st>>>(d, part);
    } else {
        if (d.c_nfast)
            k_bgemm<T, Ti::BM1, Ti::BN1, Ti::TM1, Ti::TN1, true>
                <<<(unsigned)blocks, kThreads, 0, st>>>(d, part);
        else
            k_bgemm<T, Ti::BM1, Ti::BN1, Ti::TM1, Ti::TN1, false>
                <<<(unsigned)blocks, kThreads, 0, st>>>(d, part);
    }
    if (d.nsplit > 1)
        k_bgemm_fin<T><<<(unsigned)((outs + kThreads - 1) / kThreads), kThreads, 0, st>>>(d, part);
}

template void launch_bgemm<float>(const BDesc &, void *, cudaStream_t);
template void launch_bgemm<double>(const BDesc &, void *, cudaStream_t);

}  // namespace tn

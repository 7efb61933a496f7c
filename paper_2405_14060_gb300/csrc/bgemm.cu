// Batched strided GEMM kernels (CUDA cores): contractions whose row, column
// or summed group is too small for the tensor-core tiles and whose operands
// are both too large to stream against a small one (bgemm.cuh).
//
//   k_bgemm      persistent blocks (a few per SM), each walking its share of
//                the output tiles (item, g, m tile, n tile, K split).  The A and
//                B tiles are gathered through the offset tables straight into
//                shared memory by asynchronous copies, kStages K steps ahead
//                of the multiply-adds; the pipeline runs across tile
//                boundaries, so short summed spaces (K of 8 to 32, common in
//                evidence-batched trees) still keep the memory system busy.
//                Each thread holds a TM x TN register tile whose rows and
//                columns are strided by the thread grid, so that consecutive
//                lanes store consecutive entries along C's fastest group.
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
#include <mutex>

#include "bgemm.cuh"
#include "devutil.cuh"

namespace tn {

namespace {

constexpr int kThreads = 256;
constexpr int kBK = 16;       // summed indices per pipeline stage
constexpr int kStages = 4;    // stages in flight (kStages - 1 ahead of the math)

struct TilePos {
    int64_t m0, n0, g, beta;
    int split;
};

__device__ __forceinline__ TilePos tile_pos(const BDesc &d, int64_t t, int BM, int BN) {
    const int64_t tiles_m = (d.M + BM - 1) / BM, tiles_n = (d.N + BN - 1) / BN;
    TilePos p;
    int64_t r, q = t;
    if (d.c_gfast) {
        q = div_tile(q, d.G, log2_if_pow2(d.G), r);
        p.g = r;
    }
    q = div_tile(q, tiles_m, log2_if_pow2(tiles_m), r);
    p.m0 = r * BM;
    q = div_tile(q, tiles_n, log2_if_pow2(tiles_n), r);
    p.n0 = r * BN;
    if (!d.c_gfast) {
        q = div_tile(q, d.G, log2_if_pow2(d.G), r);
        p.g = r;
    }
    q = div_tile(q, d.nbeta, log2_if_pow2(d.nbeta), r);
    p.beta = r;
    p.split = (int)q;
    return p;
}

template <typename T, int BM, int BN, int TM, int TN, bool NFAST>
__global__ void __launch_bounds__(kThreads, 2)
    k_bgemm(const __grid_constant__ BDesc d, T *part, int ntiles) {
    constexpr int MT = BM / TM, NT = BN / TN;
    static_assert(MT * NT == kThreads, "thread grid");
    // loads per thread and stage (B tiles narrower than the thread count:
    // the threads past the tile copy nothing)
    constexpr int LA = BM * kBK / kThreads, LB = (BN * kBK + kThreads - 1) / kThreads;
    static_assert(LA >= 1 && LA * kThreads == BM * kBK, "tile loads");
    constexpr int RA = BM + 1, RB = BN + 1;              // padded shared rows
    constexpr int SA = kBK * RA, SB = kBK * RB;          // per stage
    extern __shared__ __align__(16) unsigned char smraw[];
    T *As = (T *)smraw;
    T *Bs = As + kStages * SA;
    const int tid = threadIdx.x;
    const int nks = (d.kchunk + kBK - 1) / kBK;          // K steps per tile
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // fixed element mapping of this thread's tile loads: summed index within
    // the stage and shared-memory slot (bytes from the stage's base)
    int ak[LA], bk[LB], am[LA], bn[LB];
    bool bv[LB];
    uint32_t sdA[LA], sdB[LB];
#pragma unroll
    for (int r = 0; r < LA; ++r) {
        const int e = tid + kThreads * r;
        am[r] = d.a_kfast ? e / kBK : e % BM;
        ak[r] = d.a_kfast ? e % kBK : e / BM;
        sdA[r] = (uint32_t)((ak[r] * RA + am[r]) * sizeof(T));
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
        const int e = tid + kThreads * r;
        bv[r] = e < BN * kBK;
        bn[r] = bv[r] ? (d.b_kfast ? e / kBK : e % BN) : 0;
        bk[r] = bv[r] ? (d.b_kfast ? e % kBK : e / BN) : 0;
        sdB[r] = (uint32_t)((bk[r] * RB + bn[r]) * sizeof(T));
    }
    const uint32_t sA0 = (uint32_t)__cvta_generic_to_shared(As);
    const uint32_t sB0 = (uint32_t)__cvta_generic_to_shared(Bs);
    // producer state: the tile (local index) and K step being loaded next
    int p_li = 0, p_ks = 0, p_stage = 0, p_loaded = -1;
    int p_kbeg = 0, p_kend = 0;
    const T *pA = (const T *)d.A, *pB = (const T *)d.B;
    int32_t aoff[LA], boff[LB];
    auto issue = [&]() {
        if (p_li < mine) {
            if (p_li != p_loaded) {
                p_loaded = p_li;
                const TilePos tp = tile_pos(d, (int64_t)blockIdx.x + (int64_t)p_li * gridDim.x, BM, BN);
                pA = (const T *)d.A + tp.beta * d.bsa + __ldg(d.tag + tp.g);
                pB = (const T *)d.B + tp.beta * d.bsb + __ldg(d.tbg + tp.g);
                p_kbeg = tp.split * d.kchunk;
                p_kend = min(d.K, (int64_t)p_kbeg + d.kchunk);
                const int m0 = (int)tp.m0, n0 = (int)tp.n0;
#pragma unroll
                for (int r = 0; r < LA; ++r)
                    aoff[r] = m0 + am[r] < d.M ? __ldg(d.tam + m0 + am[r]) : -1;
#pragma unroll
                for (int r = 0; r < LB; ++r)
                    boff[r] = n0 + bn[r] < d.N ? __ldg(d.tbn + n0 + bn[r]) : -1;
            }
            const int k0 = p_kbeg + p_ks * kBK;
            const uint32_t sa = sA0 + (uint32_t)(p_stage * SA * sizeof(T));
            const uint32_t sb = sB0 + (uint32_t)(p_stage * SB * sizeof(T));
#pragma unroll
            for (int r = 0; r < LA; ++r) {
                const int k = k0 + ak[r];
                const bool ok = aoff[r] >= 0 && k < p_kend;
                const T *src = ok ? pA + (aoff[r] + __ldg(d.tak + k)) : pA;
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(sa + sdA[r]),
                             "l"(src), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0)
                             : "memory");
            }
#pragma unroll
            for (int r = 0; r < LB; ++r) {
                if (!bv[r]) continue;
                const int k = k0 + bk[r];
                const bool ok = boff[r] >= 0 && k < p_kend;
                const T *src = ok ? pB + (boff[r] + __ldg(d.tbk + k)) : pB;
                asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(sb + sdB[r]),
                             "l"(src), "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0)
                             : "memory");
            }
            if (++p_ks == nks) {
                p_ks = 0;
                ++p_li;
            }
            p_stage = p_stage == kStages - 1 ? 0 : p_stage + 1;
        }
        cp_async_commit();
    };
    const int im = NFAST ? tid / NT : tid % MT;
    const int in = NFAST ? tid % NT : tid / MT;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
#pragma unroll
    for (int s = 0; s < kStages - 1; ++s) issue();
    int c_li = 0, c_ks = 0, c_stage = 0;
    const bool kshort = d.nsplit == 1 && d.K <= kBK / 2;
    while (c_li < mine) {
        cp_async_wait<kStages - 2>();
        __syncthreads();
        issue();
        const T *sa = As + c_stage * SA + im;
        const T *sb = Bs + c_stage * SB + in;
        auto kstep = [&](int kk) {
            T a[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = sa[kk * RA + i * MT];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = sb[kk * RB + j * NT];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * bv[j];
        };
        if (kshort) {
            // summed space of at most half a stage: the other half is zeros
#pragma unroll
            for (int kk = 0; kk < kBK / 2; ++kk) kstep(kk);
        } else {
#pragma unroll
            for (int kk = 0; kk < kBK; ++kk) kstep(kk);
        }
        c_stage = c_stage == kStages - 1 ? 0 : c_stage + 1;
        if (++c_ks < nks) continue;
        c_ks = 0;
        // last K step of a tile: store it and start the next one
        const TilePos tp = tile_pos(d, (int64_t)blockIdx.x + (int64_t)c_li * gridDim.x, BM, BN);
        ++c_li;
        const int m0 = (int)tp.m0, n0 = (int)tp.n0;
        if (d.nsplit > 1) {
            // unscaled partials, dense [split][item][g][n][m]
            T *P = part + (((int64_t)tp.split * d.nbeta + tp.beta) * d.G + tp.g) * d.M * d.N;
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const int m = m0 + im + i * MT;
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const int n = n0 + in + j * NT;
                    if (m < d.M && n < d.N) P[(int64_t)n * d.M + m] = acc[i][j];
                    acc[i][j] = T(0);
                }
            }
            continue;
        }
        const T sca = d.mxa ? pow2neg<T>(exp_of_bits(d.mxa[tp.beta * d.mxa_bs])) : T(1);
        const T scb = d.mxb ? pow2neg<T>(exp_of_bits(d.mxb[tp.beta * d.mxb_bs])) : T(1);
        const T sc = sca * scb;
        T *Cb = (T *)d.C + tp.beta * d.bsc + __ldg(d.tcg + tp.g);
        T mx = 0;
        int32_t cn[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + in + j * NT;
            cn[j] = n < d.N ? __ldg(d.tcn + n) : -1;
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int m = m0 + im + i * MT;
            const int32_t cm = m < d.M ? __ldg(d.tcm + m) : -1;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                if (cm >= 0 && cn[j] >= 0) {
                    const T v = acc[i][j] * sc;
                    Cb[cm + cn[j]] = v;
                    mx = mx > v ? mx : v;
                }
                acc[i][j] = T(0);
            }
        }
        record_max(d.mxc, tp.beta, true, (double)mx);
    }
    cp_async_wait<0>();
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

// Tile shapes (BM x BN, thread tiles TM x TN): 0 for n > 48, 1 for
// 16 < n <= 48, 2 for 8 < n <= 16, 3 for n <= 8 (128 x 8: the 256 x 16 tile
// would leave half of every row and, for short rows, half of every column
// idle).
template <typename T>
struct Tiles;
template <>
struct Tiles<float> {
    static constexpr int BM[4] = {128, 256, 256, 128}, BN[4] = {64, 32, 16, 8};
    static constexpr int TM[4] = {8, 8, 8, 4}, TN[4] = {4, 4, 2, 1};
};
template <>
struct Tiles<double> {
    static constexpr int BM[4] = {64, 64, 128, 128}, BN[4] = {64, 32, 16, 8};
    static constexpr int TM[4] = {4, 2, 4, 4}, TN[4] = {4, 4, 2, 1};
};

template <typename T>
void tile_dims(const BDesc &d, int &bm, int &bn) {
    bm = Tiles<T>::BM[d.tile];
    bn = Tiles<T>::BN[d.tile];
}

template <typename T, int TILE>
constexpr size_t smem_bytes() {
    return (size_t)kStages * kBK *
           ((size_t)Tiles<T>::BM[TILE] + 1 + (size_t)Tiles<T>::BN[TILE] + 1) * sizeof(T);
}

// Launch one instantiation as a persistent grid: resident blocks per SM from
// the occupancy calculator (queried once), at most one block per tile.
template <typename T, int TILE, bool NFAST>
void go(const BDesc &d, T *part, int64_t ntiles, cudaStream_t st) {
    // tile counts are checked on the host to fit 31 bits
    constexpr int BM = Tiles<T>::BM[TILE], BN = Tiles<T>::BN[TILE];
    constexpr int TM = Tiles<T>::TM[TILE], TN = Tiles<T>::TN[TILE];
    constexpr size_t smem = smem_bytes<T, TILE>();
    auto kern = k_bgemm<T, BM, BN, TM, TN, NFAST>;
    static std::once_flag once;
    static int per_sm = 1, nsm = 152;
    std::call_once(once, [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kThreads, smem) ==
                cudaSuccess &&
            b > 0)
            per_sm = b;
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            n > 0)
            nsm = n;
    });
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)nsm * per_sm);
    kern<<<(unsigned)grid, kThreads, smem, st>>>(d, part, (int)ntiles);
}

}  // namespace

// Tile shape and K split; d.tile = -1 when the contraction does not fit the
// kernels' 31-bit tile and group indices.
void bgemm_configure(BDesc &d, int elem_bytes) {
    d.tile = d.N > 48 ? 0 : d.N > 16 ? 1 : d.N > 8 ? 2 : 3;
    const int bm = elem_bytes == 8 ? Tiles<double>::BM[d.tile] : Tiles<float>::BM[d.tile];
    const int bn = elem_bytes == 8 ? Tiles<double>::BN[d.tile] : Tiles<float>::BN[d.tile];
    const int64_t tiles = ((d.M + bm - 1) / bm) * ((d.N + bn - 1) / bn) * d.G * d.nbeta;
    // split the summed space when the output tiles alone leave most SMs idle
    // and every split still runs several K steps; partials stay under 1 GiB
    int64_t ns = 1;
    // (then about four waves of two resident blocks per SM, so that the last
    // wave's idle SMs weigh little)
    const int64_t want = 152LL * 3;
    if (tiles < want && d.K >= 8 * kBK) {
        ns = std::min<int64_t>((152LL * 8 + tiles - 1) / tiles, d.K / (4 * kBK));
        const int64_t outs = d.G * d.M * d.N * d.nbeta;
        while (ns > 1 && (double)ns * outs * elem_bytes > (double)(1LL << 30)) ns /= 2;
        ns = std::max<int64_t>(1, ns);
    }
    int64_t chunk = (d.K + ns - 1) / ns;
    chunk = (chunk + kBK - 1) / kBK * kBK;
    d.kchunk = std::max<int64_t>(chunk, kBK);
    d.nsplit = (int)((d.K + d.kchunk - 1) / d.kchunk);
    if (d.nsplit < 1) d.nsplit = 1;
    // the kernels count tiles and index groups in 31 bits
    if ((double)tiles * d.nsplit >= 2147483647.0 || d.M >= (1LL << 31) || d.N >= (1LL << 31) ||
        d.K >= (1LL << 31))
        d.tile = -1;
    // float data with whole K per tile and wide tiles: the tensor-core gather
    // kernel (with 32-column tiles its per-tile handoffs cost more than the
    // CUDA-core multiply-adds; measured on the 3-regular batched workload)
    d.tc = elem_bytes == 4 && d.tile >= 0 && d.nsplit == 1 && d.N > 64 && d.M >= 128 &&
           (double)tc_gather_tiles(d) < 2147483647.0;
}

size_t bgemm_scratch_bytes(const BDesc &d, int elem_bytes) {
    if (d.nsplit <= 1) return 0;
    return (size_t)d.nsplit * (size_t)(d.G * d.M * d.N * d.nbeta) * (size_t)elem_bytes;
}

int bgemm_launches(const BDesc &d) { return d.nsplit > 1 && !d.tc ? 2 : 1; }

template <typename T>
void launch_bgemm(const BDesc &d, void *scratch, cudaStream_t st) {
    const int64_t outs = d.G * d.M * d.N * d.nbeta;
    if (outs == 0) return;
    if (sizeof(T) == 4 && d.tc) {
        launch_tc_gather(d, st);
        return;
    }
    int bm, bn;
    tile_dims<T>(d, bm, bn);
    const int64_t ntiles =
        ((d.M + bm - 1) / bm) * ((d.N + bn - 1) / bn) * d.G * d.nbeta * d.nsplit;
    T *part = (T *)scratch;
    switch (d.tile * 2 + (d.c_nfast ? 1 : 0)) {
        case 0: go<T, 0, false>(d, part, ntiles, st); break;
        case 1: go<T, 0, true>(d, part, ntiles, st); break;
        case 2: go<T, 1, false>(d, part, ntiles, st); break;
        case 3: go<T, 1, true>(d, part, ntiles, st); break;
        case 4: go<T, 2, false>(d, part, ntiles, st); break;
        case 5: go<T, 2, true>(d, part, ntiles, st); break;
        case 6: go<T, 3, false>(d, part, ntiles, st); break;
        default: go<T, 3, true>(d, part, ntiles, st); break;
    }
    if (d.nsplit > 1)
        k_bgemm_fin<T><<<(unsigned)((outs + kThreads - 1) / kThreads), kThreads, 0, st>>>(d, part);
}

template void launch_bgemm<float>(const BDesc &, void *, cudaStream_t);
template void launch_bgemm<double>(const BDesc &, void *, cudaStream_t);

}  // namespace tn

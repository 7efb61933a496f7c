// Batched strided GEMM on the tensor cores (tcgen05, TF32 inputs, FP32
// accumulation), with the operands gathered in place: the contraction of
// bgemm.cuh, C[g, m, n] = sum_k A[g, m, k] B[g, k, n] over label groups,
// for float tensors in any layout.  No permutation pass: producer warps read
// each operand element through the group offset tables and write it straight
// into the 128-byte-swizzled K-major shared-memory layout that tcgen05.mma
// reads (the layout a TMA box of 32 TF32 x rows produces).
//
// One persistent CTA per SM walks its tiles (128 rows x BN columns):
//   warps 5-8  producers: asynchronous 4-byte copies of the A and B tiles of
//              each 32-index K step into a ring of shared-memory stages; a
//              thread keeps kLag steps of copies in flight, then waits for
//              the oldest, fences (generic -> async proxy) and arrives on
//              that stage's "full" barrier;
//   warp 4     MMA issuer (one thread): four tcgen05.mma kind::tf32 per
//              stage into one of two TMEM accumulators, commits free the
//              stage and, after the tile's last step, mark the accumulator
//              full;
//   warps 0-3  epilogue: tcgen05.ld of the accumulator (warp w owns rows
//              32w .. 32w+31), power-of-two scales of the operands, strided
//              stores through the C tables, per-item maximum; then the
//              accumulator is released, so tile i's epilogue overlaps tile
//              i+1's MMAs.
// Every wait is bounded in time (error flag, then the CTA drains what it
// started: copies, MMAs, and frees TMEM).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "bgemm.cuh"
#include "devutil.cuh"
#include "tcutil.cuh"

namespace tn {

namespace {

constexpr int kRows = 128;            // tile rows = TMEM lanes
constexpr int kBK = 32;               // K indices per stage: one 128-byte TF32 row
constexpr int kThr = 288;             // 4 epilogue warps, 1 MMA warp, 4 producer warps
constexpr int kProd = 128;            // producer threads
constexpr int kAB = kRows * 128;      // bytes of an A stage
constexpr int kSmemCap = 196 * 1024;  // stage ring budget

struct GParams {
    BDesc d;
    int ntiles;
    int *err;
    unsigned long long wait_ns;
};

// byte offset of element (row r, k) of a stage in the 128-byte swizzled
// K-major layout: 16-byte chunk k/4 of row r moves to chunk (k/4) xor (r mod 8)
__device__ __forceinline__ uint32_t swz(int r, int k) {
    return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ void cp4(uint32_t dst, const float *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void tile_at(const BDesc &d, int64_t t, int BN, int64_t &m0,
                                        int64_t &n0, int64_t &g, int64_t &beta) {
    const int64_t tm = (d.M + kRows - 1) / kRows, tnn = (d.N + BN - 1) / BN;
    int64_t r;
    int64_t q = div_tile(t, tm, log2_if_pow2(tm), r);
    m0 = r * kRows;
    q = div_tile(q, tnn, log2_if_pow2(tnn), r);
    n0 = r * BN;
    q = div_tile(q, d.G, log2_if_pow2(d.G), r);
    g = r;
    beta = q;
}

template <int BN>
constexpr int stages() {
    return std::min(8, kSmemCap / (kAB + BN * 128));
}

}  // namespace

template <int BN>
__global__ void __launch_bounds__(kThr, 1) k_tc_gather(const __grid_constant__ GParams p) {
    constexpr int S = stages<BN>();
    constexpr int kLag = S >= 6 ? 3 : 2;          // steps of copies a producer keeps in flight
    constexpr int kStage = kAB + BN * 128;
    const BDesc &d = p.d;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // barriers: full[S], empty[S], tfull[2], tempty[2], fin; then the TMEM slot
    uint64_t *bars = (uint64_t *)(smem + S * kStage);
    uint32_t *tslot = (uint32_t *)(bars + 2 * S + 5);
    const uint32_t sm0 = smem_u32(smem);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + S);
    const uint32_t tfull0 = smem_u32(bars + 2 * S), tempty0 = smem_u32(bars + 2 * S + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nks = (int)((d.K + kBK - 1) / kBK);
    const int mine = p.ntiles > (int)blockIdx.x
                         ? (p.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * s), "r"(kProd));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8 * a));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty0 + 8 * a), "r"(kRows));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + 2 * S + 4)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (warp >= 5) {
        // ---------------------------------------------------------- producers
        const int pid = threadIdx.x - 160, pw = pid >> 5;
        const int nq = mine * nks;
        int q = 0;
        for (; q < nq; ++q) {
            const int s = q % S;
            if (q >= S && !mbar_wait(empty0 + 8 * s, ((q / S) - 1) & 1, p.err, p.wait_ns)) break;
            const int li = q / nks, ks = q - li * nks;
            int64_t m0, n0, g, beta;
            tile_at(d, (int64_t)blockIdx.x + (int64_t)li * gridDim.x, BN, m0, n0, g, beta);
            const float *pA = (const float *)d.A + beta * d.bsa + __ldg(d.tag + g);
            const float *pB = (const float *)d.B + beta * d.bsb + __ldg(d.tbg + g);
            const int64_t k0 = (int64_t)ks * kBK;
            const uint32_t sa = sm0 + (uint32_t)(s * kStage), sb = sa + kAB;
            if (!d.a_kfast) {
                // one row per thread, consecutive threads on consecutive rows
                const int64_t m = m0 + pid;
                const int32_t ao = m < d.M ? __ldg(d.tam + m) : -1;
#pragma unroll 8
                for (int k = 0; k < kBK; ++k) {
                    const bool ok = ao >= 0 && k0 + k < d.K;
                    cp4(sa + swz(pid, k), ok ? pA + ao + __ldg(d.tak + k0 + k) : pA, ok);
                }
            } else {
                // lanes along K, each warp on every fourth row
                const bool okk = k0 + lane < d.K;
                const int32_t ko = okk ? __ldg(d.tak + k0 + lane) : 0;
#pragma unroll 8
                for (int j = 0; j < kRows / 4; ++j) {
                    const int r = pw + 4 * j;
                    const int64_t m = m0 + r;
                    const bool ok = okk && m < d.M;
                    cp4(sa + swz(r, lane), ok ? pA + __ldg(d.tam + m) + ko : pA, ok);
                }
            }
            if (!d.b_kfast) {
#pragma unroll
                for (int r = pid; r < BN; r += kProd) {
                    const int64_t n = n0 + r;
                    const int32_t bo = n < d.N ? __ldg(d.tbn + n) : -1;
#pragma unroll 8
                    for (int k = 0; k < kBK; ++k) {
                        const bool ok = bo >= 0 && k0 + k < d.K;
                        cp4(sb + swz(r, k), ok ? pB + bo + __ldg(d.tbk + k0 + k) : pB, ok);
                    }
                }
            } else {
                const bool okk = k0 + lane < d.K;
                const int32_t ko = okk ? __ldg(d.tbk + k0 + lane) : 0;
#pragma unroll 4
                for (int j = 0; j < BN / 4; ++j) {
                    const int r = pw + 4 * j;
                    const int64_t n = n0 + r;
                    const bool ok = okk && n < d.N;
                    cp4(sb + swz(r, lane), ok ? pB + __ldg(d.tbn + n) + ko : pB, ok);
                }
            }
            cp_async_commit();
            if (q >= kLag) {
                cp_async_wait<kLag>();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                 full0 + 8 * ((q - kLag) % S))
                             : "memory");
            }
        }
        // the last steps: every copy lands before the thread moves on
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int r = std::max(0, q - kLag); r < q; ++r)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * (r % S))
                         : "memory");
    } else if (warp == 4) {
        if (lane == 0) {
            // ------------------------------------------------------ MMA issuer
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                   ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
            int q = 0;
            bool ok = true;
            for (int li = 0; li < mine && ok; ++li) {
                const int a = li & 1;
                if (li >= 2 && !mbar_wait(tempty0 + 8 * a, ((li >> 1) - 1) & 1, p.err, p.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(a * BN);
                for (int ks = 0; ks < nks; ++ks, ++q) {
                    const int s = q % S;
                    if (!mbar_wait(full0 + 8 * s, (q / S) & 1, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = sm0 + (uint32_t)(s * kStage);
                    const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + kAB);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t accum = (ks | kk) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(ad + 2 * kk), "l"(bd + 2 * kk), "r"(idesc), "r"(accum));
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            empty0 + 8 * s)
                        : "memory");
                }
                if (ok)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            tfull0 + 8 * a)
                        : "memory");
            }
            // one more commit: its barrier completes once every MMA issued
            // above has finished (also after a give-up), so that TMEM is idle
            // when it is released
            (void)ok;
            const uint32_t fin = smem_u32(bars + 2 * S + 4);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(fin)
                : "memory");
            mbar_drain(fin, 0, p.err);
        }
        __syncwarp();
    } else {
        // --------------------------------------------------------- epilogue
        const int row = warp * 32 + lane;
        for (int li = 0; li < mine; ++li) {
            const int a = li & 1;
            bool have = mbar_wait(tfull0 + 8 * a, (li >> 1) & 1, p.err, p.wait_ns);
            have = __all_sync(0xffffffffu, have);
            if (!have) break;
            tc_fence_after();
            int64_t m0, n0, g, beta;
            tile_at(d, (int64_t)blockIdx.x + (int64_t)li * gridDim.x, BN, m0, n0, g, beta);
            const int64_t m = m0 + row;
            const int32_t cm = m < d.M ? __ldg(d.tcm + m) : -1;
            const float sca = d.mxa ? pow2neg<float>(exp_of_bits(d.mxa[beta * d.mxa_bs])) : 1.f;
            const float scb = d.mxb ? pow2neg<float>(exp_of_bits(d.mxb[beta * d.mxb_bs])) : 1.f;
            const float sc = sca * scb;
            float *Cb = (float *)d.C + beta * d.bsc + __ldg(d.tcg + g);
            float mx = 0.f;
            for (int c = 0; c < BN / 32; ++c) {
                if (n0 + c * 32 >= d.N) break;   // warp-uniform: no columns left
                uint32_t r[32];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * BN + c * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                    "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
                    "%26, %27, %28, %29, %30, %31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                      "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                      "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                      "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (cm >= 0) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t n = n0 + c * 32 + j;
                        if (n < d.N) {
                            const float v = __uint_as_float(r[j]) * sc;
                            Cb[cm + __ldg(d.tcn + n)] = v;
                            mx = fmaxf(mx, v);
                        }
                    }
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * a) : "memory");
            record_max(d.mxc, beta, true, (double)mx);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * BN));
}

namespace {

template <int BN>
void go_tc(const GParams &gp, cudaStream_t st) {
    constexpr int S = stages<BN>();
    constexpr size_t smem = (size_t)S * (kAB + BN * 128) + 1024 + 256;
    static std::once_flag once;
    static int nsm = 152;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_tc_gather<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            n > 0)
            nsm = n;
    });
    const int grid = std::min(gp.ntiles, nsm);
    k_tc_gather<BN><<<grid, kThr, smem, st>>>(gp);
}

int gather_bn(int64_t N) { return N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256; }

}  // namespace

int64_t tc_gather_tiles(const BDesc &d) {
    const int bn = gather_bn(d.N);
    return ((d.M + kRows - 1) / kRows) * ((d.N + bn - 1) / bn) * d.G * d.nbeta;
}

void launch_tc_gather(const BDesc &d, cudaStream_t st) {
    GParams gp;
    gp.d = d;
    gp.ntiles = (int)tc_gather_tiles(d);
    gp.err = d.err;
    gp.wait_ns = TC_WAIT_NS;
    if (const char *w = getenv("TN_TEST_TC_WAIT_NS")) gp.wait_ns = strtoull(w, nullptr, 10);
    if (gp.ntiles <= 0) return;
    switch (gather_bn(d.N)) {
        case 32: go_tc<32>(gp, st); break;
        case 64: go_tc<64>(gp, st); break;
        case 128: go_tc<128>(gp, st); break;
        default: go_tc<256>(gp, st); break;
    }
}

}  // namespace tn

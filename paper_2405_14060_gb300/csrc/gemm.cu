// Dense pairwise contractions as batched GEMMs (the paper's "each pairwise
// contraction can be decomposed into BLAS operations", Sec. Tensor networks),
// written for sm_103a:
//
//   k_permute    operand preparation: a strided tensor to GEMM form
//                [batch][rows][K] (K contiguous), with the per-item exact
//                power-of-two rescale and the conversion to the GEMM input
//                type; also used to scatter a GEMM result into a tensor's
//                layout while recording its per-item maximum.
//   k_tc_gemm    tcgen05 tensor-core GEMM: D = X Y^T per batch, X and Y
//                K-major, TF32 (kind::tf32) or BF16 (kind::f16) inputs staged
//                by TMA (128-byte swizzle) through a 4-stage mbarrier
//                pipeline, FP32 accumulators in TMEM (two 128 x 256 buffers
//                per CTA), epilogue through tcgen05.ld.  One thread issues
//                TMA, one issues MMAs, four warps drain TMEM; persistent over
//                tiles for short K, so that a tile's epilogue overlaps the
//                next tile's MMAs.
//   k_simt_gemm  CUDA-core tiled GEMM for FP32 and FP64.
//
// Every mbarrier wait is bounded in time: a wait that exceeds ~2 s sets the
// error flag and the CTA skips the rest of its work.  Before it frees its
// TMEM and exits it waits (bounded again) for the asynchronous work it has
// already started: the TMA transfers of the last stages it issued and, via a
// final commit, every MMA it issued.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "devutil.cuh"
#include "gemm.cuh"
#include "tcutil.cuh"

namespace tn {

// ------------------------------------------------------------- permute

template <typename TI, int OT>
__device__ __forceinline__ void store_conv(void *out, int64_t i, TI x);

// Element-wise form: one element per thread and step, in the input type (the
// scale is an exact power of two).
template <typename TI, int OT>
__global__ void __launch_bounds__(256) k_permute(const __grid_constant__ PDesc p, int64_t per) {
    // blockIdx.y = batch item when the outermost dimension is the batch label
    // and maxima are recorded (per = entries per item); else blockIdx.y = 0
    // and per = total.
    const int64_t item = blockIdx.y;
    TI mxv = 0;
    constexpr int U = 8;
    const TI *in = (const TI *)p.in;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < per; i0 += stride * U) {
        int64_t oi[U], oo[U], beta[U];
        TI v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int64_t i = i0 + u * stride;
            const int64_t idx = item * per + (i < per ? i : 0);
            oi[u] = 0;
            oo[u] = 0;
            beta[u] = 0;
            if (p.pow2) {
                for (int d = 0; d < p.nd; ++d) {
                    int64_t dg = (idx >> p.sh[d]) & (int64_t)(p.sz[d] - 1);
                    oi[u] += dg * p.sin[d];
                    oo[u] += dg * p.sout[d];
                    if (d == p.beta_dim) beta[u] = dg;
                }
            } else {
                int64_t r = idx;
                for (int d = p.nd - 1; d >= 0; --d) {
                    int64_t dg = r % p.sz[d];
                    r /= p.sz[d];
                    oi[u] += dg * p.sin[d];
                    oo[u] += dg * p.sout[d];
                    if (d == p.beta_dim) beta[u] = dg;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = in[oi[u]];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i0 + u * stride >= per) continue;
            TI x = v[u];
            if (p.mxi) x *= pow2neg<TI>(exp_of_bits(p.mxi[beta[u] * p.mxi_bs]));
            store_conv<TI, OT>(p.out, oo[u], x);
            mxv = mxv > x ? mxv : x;
        }
    }
    if (p.mxo) block_max_atomic(p.mxo + item, (double)mxv);
}

template <typename TI, int OT>
__device__ __forceinline__ void store_conv(void *out, int64_t i, TI x) {
    if (OT == E_F64) ((double *)out)[i] = (double)x;
    else if (OT == E_F32) ((float *)out)[i] = (float)x;
    else ((__nv_bfloat16 *)out)[i] = __float2bfloat16_rn((float)x);
}

// Tiled form: each block walks a contiguous range of tiles (up to PT_MAXN
// entries each, input and output runs of at least 32 entries) through three
// shared-memory buffers: while tile q is written out, the asynchronous copies
// of tiles q + 1 and q + 2 are in flight, and one barrier per tile both
// publishes a landed tile and frees the buffer of the previous one.  Thread 0
// advances the tiles' base offsets digit by digit, three tiles ahead, and
// publishes them in shared memory.  Loads follow the input order (t.vin
// inputs per 16-byte copy when the plan allows), stores the output order
// (t.vec outputs per 16-byte store, their shared-memory slots read as one
// vector of 16-bit integers).
template <typename TI, int OT>
__global__ void __launch_bounds__(256, 4) k_permute_tiled(const __grid_constant__ PDesc p,
                                                       int64_t per_item) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int64_t sbase[4][3];   // per tile (mod 4): input base, output base, item
    const PTile &t = p.tl;
    const int n = t.tn;
    const int nbuf = t.nbuf, swz = t.swz;
    TI *sm0 = (TI *)smraw;
    const int64_t item = blockIdx.y;
    const int32_t *tin = t.ttab, *tout = t.ttab + n;
    const uint16_t *slot = (const uint16_t *)(t.ttab + 2 * n);
    const TI *in = (const TI *)p.in;
    TI mxv = 0;
    // this block's tiles [q0, q1)
    const int64_t q0 = per_item * blockIdx.x / gridDim.x;
    const int64_t q1 = per_item * (blockIdx.x + 1) / gridDim.x;
    // digits of the last published tile (thread 0 only)
    int32_t dg[MAXD];
    int64_t cbi = 0, cbo = 0;
    if (threadIdx.x == 0) {
        uint32_t g = (uint32_t)(item * per_item + q0);
        for (int k = t.nrest - 1; k >= 0; --k) {
            uint32_t v;
            if (t.rsh[k] >= 0) {
                v = g & (uint32_t)(t.rsz[k] - 1);
                g >>= t.rsh[k];
            } else {
                v = g % (uint32_t)t.rsz[k];
                g /= (uint32_t)t.rsz[k];
            }
            dg[k] = (int32_t)v;
            cbi += (int64_t)v * t.rin[k];
            cbo += (int64_t)v * t.rout[k];
        }
    }
    // thread 0: publish the bases of tile q (called for q0, q0 + 1, ... in order)
    auto publish = [&](int64_t q) {
        if (threadIdx.x != 0 || q >= q1) return;
        if (q > q0) {
            for (int k = t.nrest - 1; k >= 0; --k) {
                cbi += t.rin[k];
                cbo += t.rout[k];
                if (++dg[k] < t.rsz[k]) break;
                cbi -= t.rin[k] * t.rsz[k];
                cbo -= t.rout[k] * t.rsz[k];
                dg[k] = 0;
            }
        }
        const int s = (int)(q & 3);
        sbase[s][0] = cbi;
        sbase[s][1] = cbo;
        sbase[s][2] = t.rest_beta >= 0 ? dg[t.rest_beta] : 0;
    };
    const bool vin = t.vin > 0 && ((uintptr_t)p.in & 15) == 0;
    // copies of tile q into buffer buf (an empty group past the range)
    auto issue = [&](int64_t q, int buf) {
        if (q < q1) {
            const int64_t bi = sbase[q & 3][0];
            const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(sm0 + buf * nbuf);
            if (vin) {
                constexpr int GI = 16 / (int)sizeof(TI);
                for (int e = threadIdx.x * GI; e < n; e += 256 * GI)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                     s0 + (uint32_t)(pt_slot<sizeof(TI)>(e, swz) * sizeof(TI))),
                                 "l"(in + bi + __ldg(tin + e))
                                 : "memory");
            } else {
                for (int e = threadIdx.x; e < n; e += 256)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                                     s0 + (uint32_t)(pt_slot<sizeof(TI)>(e, swz) * sizeof(TI))),
                                 "l"(in + bi + __ldg(tin + e)), "n"(sizeof(TI))
                                 : "memory");
            }
        }
        cp_async_commit();
    };
    const bool vec = t.vec > 0 && ((uintptr_t)p.out & 15) == 0;
    publish(q0);
    publish(q0 + 1);
    publish(q0 + 2);
    __syncthreads();
    issue(q0, 0);
    issue(q0 + 1, 1);
    int buf = 0;
    for (int64_t q = q0; q < q1; ++q) {
        cp_async_wait<1>();
        // every thread's copies of tile q landed, every thread is done with
        // tile q - 1 (its buffer is free), and the bases of q + 2 are visible
        __syncthreads();
        issue(q + 2, buf == 0 ? 2 : buf - 1);
        publish(q + 3);
        const int64_t bo = sbase[q & 3][1], beta = sbase[q & 3][2];
        const TI sc = p.mxi ? pow2neg<TI>(exp_of_bits(p.mxi[beta * p.mxi_bs])) : TI(1);
        const TI *sm = sm0 + buf * nbuf;
        if (vec) {
            constexpr int G = OT == E_F64 ? 2 : OT == E_F32 ? 4 : 8;
            for (int e0 = threadIdx.x * G; e0 < n; e0 += 256 * G) {
                uint16_t sl[G];
                if (G == 8) *(uint4 *)sl = __ldg((const uint4 *)(slot + e0));
                else if (G == 4) *(uint2 *)sl = __ldg((const uint2 *)(slot + e0));
                else *(uint32_t *)sl = __ldg((const uint32_t *)(slot + e0));
                TI x[G];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    x[j] = sm[sl[j]] * sc;
                    mxv = mxv > x[j] ? mxv : x[j];
                }
                const int64_t o = bo + __ldg(tout + e0);
                if (OT == E_BF16) {
                    uint4 v;
                    uint32_t *w = (uint32_t *)&v;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        __nv_bfloat162 h = __floats2bfloat162_rn((float)x[2 * j], (float)x[2 * j + 1]);
                        w[j] = *(uint32_t *)&h;
                    }
                    *(uint4 *)((__nv_bfloat16 *)p.out + o) = v;
                } else if (OT == E_F32) {
                    *(float4 *)((float *)p.out + o) =
                        make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
                } else {
                    *(double2 *)((double *)p.out + o) = make_double2((double)x[0], (double)x[1]);
                }
            }
        } else {
            for (int e = threadIdx.x; e < n; e += 256) {
                TI x = sm[__ldg(slot + e)] * sc;
                store_conv<TI, OT>(p.out, bo + __ldg(tout + e), x);
                mxv = mxv > x ? mxv : x;
            }
        }
        buf = buf == 2 ? 0 : buf + 1;
    }
    cp_async_wait<0>();
    if (p.mxo) block_max_atomic(p.mxo + item, (double)mxv);
}

void plan_permute_tiles(PDesc &p, std::vector<int32_t> &tab) {
    p.tl.tn = 0;
    tab.clear();
    if (p.nd < 2 || p.total < 8192 || p.total / 64 >= (1LL << 31)) return;
    struct D { int64_t sz, sin, sout; bool beta; };
    std::vector<D> d;
    for (int i = 0; i < p.nd; ++i) d.push_back({p.sz[i], p.sin[i], p.sout[i], i == p.beta_dim});
    constexpr int64_t RUN = 32;
    std::vector<char> in_u(d.size(), 0);
    int64_t n = 1;
    bool full = false;
    // dims below `lim` on one side (lim < 0: the next input-fastest dims
    // until the tile holds 2048 entries), up to `cap` entries in the tile (a
    // dim that would pass it is split; at PT_MAXN the tile is full)
    auto add_below = [&](bool by_in, int64_t lim, int64_t cap) {
        while (!full && (lim > 0 || n < 2048)) {
            int best = -1;
            for (int i = 0; i < (int)d.size(); ++i) {
                if (in_u[i] || d[i].beta || d[i].sz < 2) continue;
                int64_t st = by_in ? d[i].sin : d[i].sout;
                if (lim > 0 && st >= lim) continue;
                if (best < 0 || st < (by_in ? d[best].sin : d[best].sout)) best = i;
            }
            if (best < 0) return;
            if (n * d[best].sz <= cap) {
                in_u[best] = 1;
                n *= d[best].sz;
                continue;
            }
            int64_t lo = cap / n;
            while (lo >= 2 && d[best].sz % lo) --lo;
            if (lo >= 2) {
                D hi{d[best].sz / lo, d[best].sin * lo, d[best].sout * lo, false};
                D lw{lo, d[best].sin, d[best].sout, false};
                d[best] = hi;
                d.insert(d.begin() + best + 1, lw);
                in_u.insert(in_u.begin() + best + 1, 1);
                n *= lo;
            }
            if (cap >= PT_MAXN) full = true;
            return;
        }
    };
    // the input's contiguous side first, but at most 128 entries of it, so
    // that a long contiguous input run (a plain transpose) still leaves room
    // for at least 32 contiguous outputs; then the output's; then more of
    // the input's
    add_below(true, RUN, 4 * RUN);
    add_below(false, RUN, PT_MAXN);
    add_below(true, -1, PT_MAXN);
    if (n < 256) return;
    std::vector<int> U;
    for (int i = 0; i < (int)d.size(); ++i)
        if (in_u[i]) U.push_back(i);
    auto order_by = [&](bool by_in) {
        std::vector<int> o = U;
        std::sort(o.begin(), o.end(), [&](int a, int b) {
            return by_in ? d[a].sin < d[b].sin : d[a].sout < d[b].sout;
        });
        return o;   // fastest digit first
    };
    std::vector<int> oi = order_by(true), oo = order_by(false);
    // digit vector -> index in the input order
    std::vector<int64_t> wi(d.size(), 0);
    {
        int64_t w = 1;
        for (int i : oi) {
            wi[i] = w;
            w *= d[i].sz;
        }
    }
    // input offsets [n], output offsets [n], then the 16-bit slots [n]
    tab.assign((size_t)(2 * n + (n + 1) / 2), 0);
    for (int64_t e = 0; e < n; ++e) {
        int64_t r = e, off = 0;
        for (int i : oi) {
            int64_t dg = r % d[i].sz;
            r /= d[i].sz;
            off += dg * d[i].sin;
        }
        if (off >= (1LL << 31)) {
            tab.clear();
            return;
        }
        tab[e] = (int32_t)off;
    }
    std::vector<int> ein_of((size_t)n);
    for (int64_t e = 0; e < n; ++e) {
        int64_t r = e, off = 0, ein = 0;
        for (int i : oo) {
            int64_t dg = r % d[i].sz;
            r /= d[i].sz;
            off += dg * d[i].sout;
            ein += dg * wi[i];
        }
        if (off >= (1LL << 31)) {
            tab.clear();
            return;
        }
        tab[n + e] = (int32_t)off;
        ein_of[e] = (int)ein;
    }
    PTile &t = p.tl;
    t.nrest = 0;
    t.rest_beta = -1;
    t.ntiles = 1;
    for (int i = 0; i < (int)d.size(); ++i) {
        if (in_u[i]) continue;
        if (t.nrest >= MAXD) {
            tab.clear();
            return;
        }
        if (d[i].beta) t.rest_beta = t.nrest;
        t.rsz[t.nrest] = (int32_t)d[i].sz;
        t.rsh[t.nrest] = (d[i].sz & (d[i].sz - 1)) ? -1 : __builtin_ctzll((unsigned long long)d[i].sz);
        t.rin[t.nrest] = d[i].sin;
        t.rout[t.nrest] = d[i].sout;
        t.ntiles *= d[i].sz;
        ++t.nrest;
    }
    // per-item maxima need the batch dim outermost (one item per grid row)
    if ((p.mxo && t.rest_beta > 0) || t.ntiles >= (1LL << 31)) {
        tab.clear();
        return;
    }
    t.tn = (int)n;
    t.ttab = nullptr;   // device copy of `tab`, set by the caller
    // 16-byte stores: every aligned group of G output-ordered entries is
    // contiguous and starts on a multiple of G elements in every tile
    t.vec = 0;
    {
        const int G = p.out_type == E_F64 ? 2 : p.out_type == E_F32 ? 4 : 8;
        bool ok = n % G == 0;
        for (int64_t e0 = 0; ok && e0 < n; e0 += G) {
            const int32_t o = tab[n + e0];
            ok = o % G == 0;
            for (int j = 1; ok && j < G; ++j) ok = tab[n + e0 + j] == o + j;
        }
        for (int k = 0; ok && k < t.nrest; ++k) ok = t.rout[k] % G == 0;
        if (ok) t.vec = G;
    }
    // 16-byte input copies: the same condition on the input-ordered entries
    t.vin = 0;
    {
        const int G = p.in_type == E_F64 ? 2 : 4;
        bool ok = n % G == 0;
        for (int64_t e0 = 0; ok && e0 < n; e0 += G) {
            const int32_t o = tab[e0];
            ok = o % G == 0;
            for (int j = 1; ok && j < G; ++j) ok = tab[e0 + j] == o + j;
        }
        for (int k = 0; ok && k < t.nrest; ++k) ok = t.rin[k] % G == 0;
        if (ok) t.vin = G;
    }
    // shared-memory layout: the one whose reads of a tile (output order,
    // t.vec entries per thread, or one) take the fewest wavefronts
    {
        const int esz = p.in_type == E_F64 ? 8 : 4;
        const int G = t.vec > 0 ? t.vec : 1;
        auto slot_of = [&](int e, int swz) {
            return esz == 8 ? pt_slot<8>(e, swz) : pt_slot<4>(e, swz);
        };
        int64_t best = -1;
        std::vector<int> sl((size_t)n);
        for (int swz = 0; swz < PT_NSWZ; ++swz) {
            for (int64_t e = 0; e < n; ++e) sl[e] = slot_of(ein_of[e], swz);
            int64_t waves = 0;
            for (int64_t b = 0; b < n; b += 256 * G)
                for (int w = 0; w < 8; ++w)
                    for (int j = 0; j < G; ++j) {
                        // one warp-wide shared load: per bank, the distinct words
                        int cnt[32] = {0};
                        int64_t seen[32][32];
                        for (int l = 0; l < 32; ++l) {
                            const int64_t e = b + (int64_t)(w * 32 + l) * G + j;
                            if (e >= n) continue;
                            const int64_t word = (int64_t)sl[e] * (esz / 4);
                            const int bank = (int)(word & 31);
                            bool dup = false;
                            for (int k = 0; k < cnt[bank]; ++k) dup = dup || seen[bank][k] == word;
                            if (!dup) seen[bank][cnt[bank]++] = word;
                        }
                        int mx = 0;
                        for (int k = 0; k < 32; ++k) mx = std::max(mx, cnt[k]);
                        waves += mx;
                    }
            if (best < 0 || waves < best) {
                best = waves;
                t.swz = swz;
            }
        }
        t.nbuf = pt_nbuf((int)n, t.swz);
        uint16_t *s16 = (uint16_t *)(tab.data() + 2 * n);
        for (int64_t e = 0; e < n; ++e) s16[e] = (uint16_t)slot_of(ein_of[e], t.swz);
    }
}

void launch_permute(const PDesc &p, cudaStream_t st) {
    if (p.total <= 0) return;
    if (p.tl.tn > 0 && p.tl.ttab) {
        int nitems = (p.mxo && p.tl.rest_beta == 0) ? p.tl.rsz[0] : 1;
        int64_t per = p.tl.ntiles / nitems;
        // three tile buffers; as many blocks per SM as shared memory holds
        size_t sm = 3 * (size_t)p.tl.nbuf * (p.in_type == E_F64 ? 8 : 4);
        const int64_t bps = std::max<int64_t>(1, std::min<int64_t>(8, (227 * 1024) / (sm + 1024)));
        int64_t cap = std::max<int64_t>(1, (152LL * bps) / nitems);
        dim3 grid((unsigned)std::max<int64_t>(1, std::min(per, cap)), (unsigned)nitems, 1);
        static std::once_flag once;
        std::call_once(once, [] {
            const int mx = 3 * pt_nbuf(PT_MAXN, 0) * 8;
            cudaFuncSetAttribute(k_permute_tiled<double, E_F64>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_permute_tiled<float, E_F32>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_permute_tiled<float, E_BF16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        });
        if (p.in_type == E_F64) k_permute_tiled<double, E_F64><<<grid, 256, sm, st>>>(p, per);
        else if (p.out_type == E_F32) k_permute_tiled<float, E_F32><<<grid, 256, sm, st>>>(p, per);
        else k_permute_tiled<float, E_BF16><<<grid, 256, sm, st>>>(p, per);
        return;
    }
    int nitems = 1;
    if (p.mxo && p.beta_dim == 0) nitems = p.sz[0];
    int64_t per = p.total / nitems;
    dim3 grid = item_grid((per + 3) / 4, nitems);
    if (p.in_type == E_F64) k_permute<double, E_F64><<<grid, 256, 0, st>>>(p, per);
    else if (p.out_type == E_F32) k_permute<float, E_F32><<<grid, 256, 0, st>>>(p, per);
    else k_permute<float, E_BF16><<<grid, 256, 0, st>>>(p, per);
}

// ------------------------------------------------------------ tcgen05 GEMM

constexpr int TC_BM = 128, TC_BN = 256, TC_STAGES = 4;
constexpr int TC_XBYTES = TC_BM * 128, TC_YBYTES = TC_BN * 128;    // one 128-byte K slab
constexpr int TC_SMEM = TC_STAGES * (TC_XBYTES + TC_YBYTES) + 1024 + 256;
constexpr int TC_THREADS = 192;   // warps 0-3 epilogue, warp 4 MMA issuer, warp 5 TMA producer

struct TCParams {
    int64_t R, C, ldd, bsd;
    int64_t ntn, ntm;           // column / row tiles; tiles = batch x rows x columns
    int64_t ntiles;
    const unsigned long long *mxsx;   // scale of X applied to D (NULL: none)
    int kt;                     // number of 128-byte K slabs
    float *D;
    unsigned long long *mxd;
    int64_t beta_div_batch, beta_div_row;
    int *err;
    unsigned long long wait_ns;   // limit of the producer's and the MMA issuer's waits
};

// Tile t: batch item, first row, first column.  Within a batch item the
// row tiles go in groups of TC_GROUP, and a group's tiles run rows fastest,
// so that the tiles processed together read a few row panels of X and a few
// column panels of Y (which then stay in L2) rather than all of Y.
constexpr int TC_GROUP = 8;
__device__ __forceinline__ void tc_tile(const TCParams &p, int64_t t, int &bz, int64_t &m0,
                                        int64_t &n0) {
    const int64_t per_b = p.ntn * p.ntm;
    bz = (int)(t / per_b);
    const int64_t rem = t - (int64_t)bz * per_b;
    const int64_t per_g = (int64_t)TC_GROUP * p.ntn;
    const int64_t grp = rem / per_g, loc = rem - grp * per_g;
    const int64_t rows = min((int64_t)TC_GROUP, p.ntm - grp * TC_GROUP);
    m0 = (grp * TC_GROUP + loc % rows) * TC_BM;
    n0 = (loc / rows) * TC_BN;
}

// Persistent: CTA b takes tiles b, b + grid, ...  The TMA warp fills a ring
// of TC_STAGES K slabs (X and Y tiles, 128-byte swizzle) across tile
// boundaries; the MMA warp accumulates tile i into one of two 256-column TMEM
// buffers (i & 1) while the four epilogue warps drain the other one, so a
// tile's TMEM -> global epilogue overlaps the next tile's MMAs.  Every wait
// is bounded: on a timeout the error flag is set, the producer waits for the
// copies it issued, the MMA warp for the MMAs it issued, and TMEM is freed.
template <int BF16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap ty,
              const __grid_constant__ TCParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sX = smem;
    uint8_t *sY = smem + TC_STAGES * TC_XBYTES;
    // barriers: full[S], empty[S], tfull[2], tempty[2], fin; then the TMEM slot
    uint64_t *bars = (uint64_t *)(sY + TC_STAGES * TC_YBYTES);
    uint32_t *tslot = (uint32_t *)(bars + 2 * TC_STAGES + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + TC_STAGES),
                   tfull0 = smem_u32(bars + 2 * TC_STAGES),
                   tempty0 = smem_u32(bars + 2 * TC_STAGES + 2),
                   fin = smem_u32(bars + 2 * TC_STAGES + 4);
    const int mine = p.ntiles > (int64_t)blockIdx.x
                         ? (int)((p.ntiles - 1 - (int64_t)blockIdx.x) / gridDim.x) + 1
                         : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * s));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * s));
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8 * a));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty0 + 8 * a),
                         "r"(TC_BM));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fin));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&tx) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(&ty) : "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(2 * TC_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int KT = p.kt;
    if (warp == 5) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            int q = 0;   // K slabs issued so far (all tiles)
            bool ok = true;
            for (int li = 0; li < mine && ok; ++li) {
                int bz;
                int64_t m0, n0;
                tc_tile(p, (int64_t)blockIdx.x + (int64_t)li * gridDim.x, bz, m0, n0);
                for (int kt = 0; kt < KT; ++kt, ++q) {
                    const int s = q % TC_STAGES;
                    if (q >= TC_STAGES &&
                        !mbar_wait(empty0 + 8 * s, ((q / TC_STAGES) - 1) & 1, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = full0 + 8 * s;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                 "r"(TC_XBYTES + TC_YBYTES)
                                 : "memory");
                    const int kx = kt * (BF16 ? 64 : 32);
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(sX + s * TC_XBYTES)),
                        "l"(&tx), "r"(fb), "r"(kx), "r"((int)m0), "r"(bz)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(sY + s * TC_YBYTES)),
                        "l"(&ty), "r"(fb), "r"(kx), "r"((int)n0), "r"(bz)
                        : "memory");
                }
            }
            // the last transfers issued land before the CTA exits (already
            // the case when the MMA warp consumed them; it may have given up)
            for (int r = q > TC_STAGES ? q - TC_STAGES : 0; r < q; ++r)
                mbar_drain(full0 + 8 * (r % TC_STAGES), (r / TC_STAGES) & 1, p.err);
        }
        __syncwarp();
    } else if (warp == 4) {
        if (lane == 0) {
            // ------------------------------------------------- MMA issuer
            // D[128 x 256] (+)= X[128 x K] * Y[256 x K]^T, 4 MMAs of 32 bytes of K per slab
            const uint32_t idesc = (1u << 4) |                               // D: F32
                                   ((BF16 ? 1u : 2u) << 7) |                 // A: BF16 / TF32
                                   ((BF16 ? 1u : 2u) << 10) |                // B: BF16 / TF32
                                   ((uint32_t)(TC_BN >> 3) << 17) |          // N
                                   ((uint32_t)(TC_BM >> 4) << 24);           // M
            int q = 0;
            bool ok = true;
            for (int li = 0; li < mine && ok; ++li) {
                const int a = li & 1;
                // the epilogue has drained this TMEM buffer (tile li - 2)
                if (li >= 2 && !mbar_wait(tempty0 + 8 * a, ((li >> 1) - 1) & 1, p.err, p.wait_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc_t = tmem + (uint32_t)(a * TC_BN);
                for (int kt = 0; kt < KT; ++kt, ++q) {
                    const int s = q % TC_STAGES;
                    if (!mbar_wait(full0 + 8 * s, (q / TC_STAGES) & 1, p.err, p.wait_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = sdesc_sw128(smem_u32(sX + s * TC_XBYTES));
                    const uint64_t bd = sdesc_sw128(smem_u32(sY + s * TC_YBYTES));
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t accum = (kt | kk) ? 1u : 0u;
                        if (BF16)
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                    acc_t),
                                "l"(ad + 2 * kk), "l"(bd + 2 * kk), "r"(idesc), "r"(accum));
                        else
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                    acc_t),
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
            // completes once every MMA issued above has finished (also after
            // a give-up), so that TMEM is idle when it is released
            (void)ok;
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(fin)
                : "memory");
            mbar_drain(fin, 0, p.err);
        }
        __syncwarp();
    } else {
        // ----------------------------------------------------- epilogue
        // warp w drains TMEM lanes 32w..32w+31 (rows of the tile)
        const float sxs = p.mxsx ? pow2neg<float>(exp_of_bits(*p.mxsx)) : 1.f;
        for (int li = 0; li < mine; ++li) {
            const int a = li & 1;
            bool have = mbar_wait(tfull0 + 8 * a, (li >> 1) & 1, p.err, p.wait_ns);
            have = __all_sync(0xffffffffu, have);
            if (!have) break;
            tc_fence_after();
            int bz;
            int64_t m0, n0;
            tc_tile(p, (int64_t)blockIdx.x + (int64_t)li * gridDim.x, bz, m0, n0);
            const int64_t row = m0 + warp * 32 + lane;
            float mx = 0;
            float *drow = p.D + (int64_t)bz * p.bsd + row * p.ldd;
            for (int ch = 0; ch < TC_BN / 32; ++ch) {
                if (n0 + ch * 32 >= p.C) break;   // warp-uniform: no columns left
                uint32_t r[32];
                const uint32_t ta =
                    tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * TC_BN + ch * 32);
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
                const int64_t c0 = n0 + ch * 32;
                if (row < p.R) {
                    if (c0 + 32 <= p.C && (p.ldd % 4) == 0) {
                        float4 *dst = (float4 *)(drow + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float4 v;
                            v.x = __uint_as_float(r[4 * j + 0]) * sxs;
                            v.y = __uint_as_float(r[4 * j + 1]) * sxs;
                            v.z = __uint_as_float(r[4 * j + 2]) * sxs;
                            v.w = __uint_as_float(r[4 * j + 3]) * sxs;
                            dst[j] = v;
                            mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
                        }
                    } else {
                        for (int j = 0; j < 32 && c0 + j < p.C; ++j) {
                            const float v = __uint_as_float(r[j]) * sxs;
                            drow[c0 + j] = v;
                            mx = fmaxf(mx, v);
                        }
                    }
                }
            }
            // this TMEM buffer may take the MMAs of tile li + 2
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8 * a) : "memory");
            const int64_t beta = p.beta_div_batch > 0 ? (int64_t)bz / p.beta_div_batch
                                 : p.beta_div_row > 0 ? (row < p.R ? row : p.R - 1) / p.beta_div_row
                                                      : 0;
            record_max(p.mxd, beta, row < p.R, (double)mx);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * TC_BN));
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

bool tc_gemm_supported(const GDesc &g) {
    int es = g.xtype == E_BF16 ? 2 : 4;
    if (g.xtype == E_F64) return false;
    if (((uintptr_t)g.X | (uintptr_t)g.Y) & 15) return false;
    if ((g.ldx * es) % 16 || (g.ldy * es) % 16) return false;
    if (g.batch > 1 && ((g.bsx * es) % 16 || (g.bsy * es) % 16)) return false;
    if (g.R > (1LL << 31) - TC_BM || g.C > (1LL << 31) - TC_BN) return false;
    if (((g.C + TC_BN - 1) / TC_BN) * ((g.R + TC_BM - 1) / TC_BM) * g.batch >= (1LL << 31)) return false;
    if (g.K < 1) return false;
    return encode_fn() != nullptr;
}

static bool make_map(CUtensorMap *m, const void *base, int64_t K, int64_t rows, int64_t batch,
                     int64_t ld, int64_t bs, int es, bool bf16, int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)((batch > 1 ? bs : rows * ld) * es)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                             3, (void *)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_tc_gemm(const GDesc &g, int *err_flag, cudaStream_t st) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_tc_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    });
    bool bf16 = g.xtype == E_BF16;
    int es = bf16 ? 2 : 4;
    CUtensorMap mx, my;
    if (!make_map(&mx, g.X, g.K, g.R, g.batch, g.ldx, g.bsx, es, bf16, TC_BM) ||
        !make_map(&my, g.Y, g.K, g.C, g.batch, g.ldy, g.bsy, es, bf16, TC_BN))
        return cudaErrorInvalidValue;
    TCParams p;
    p.R = g.R;
    p.C = g.C;
    p.ldd = g.ldd;
    p.bsd = g.bsd;
    int kel = 128 / es;
    p.kt = (int)((g.K + kel - 1) / kel);
    p.D = (float *)g.D;
    p.mxd = g.mxd;
    p.mxsx = g.mxsx;
    p.beta_div_batch = g.beta_div_batch;
    p.beta_div_row = g.beta_div_row;
    p.err = err_flag;
    // test hook: a shorter limit for the pipeline's waits (nanoseconds), so
    // that tests can make them give up without any fault
    p.wait_ns = TC_WAIT_NS;
    if (const char *w = getenv("TN_TEST_TC_WAIT_NS")) p.wait_ns = strtoull(w, nullptr, 10);
    p.ntn = (g.C + TC_BN - 1) / TC_BN;
    p.ntm = (g.R + TC_BM - 1) / TC_BM;
    p.ntiles = p.ntn * p.ntm * g.batch;
    if (p.ntiles >= (1LL << 31)) return cudaErrorInvalidConfiguration;
    // short K (at most 64 slabs): persistent, one CTA per SM (its shared
    // memory and the whole TMEM), each tile's epilogue overlapping the next
    // tile's MMAs; long K: one tile per CTA (the epilogue is a small part of
    // the tile, and CTAs started in tile order keep the concurrently read
    // operand panels close together in L2, where persistent CTAs drift apart
    // over hundreds of K slabs; measured on the batched workload's nodes)
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, n = 0;
        nsm = (cudaGetDevice(&dev) == cudaSuccess &&
               cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
                  ? n
                  : 152;
    }
    dim3 grid((unsigned)(p.kt <= 64 ? std::min<int64_t>(p.ntiles, nsm) : p.ntiles), 1, 1);
    if (bf16) k_tc_gemm<1><<<grid, TC_THREADS, TC_SMEM, st>>>(mx, my, p);
    else k_tc_gemm<0><<<grid, TC_THREADS, TC_SMEM, st>>>(mx, my, p);
    return cudaGetLastError();
}

// ------------------------------------------------------------- SIMT GEMM

template <typename T>
__global__ void __launch_bounds__(256) k_simt_gemm(const __grid_constant__ GDesc g) {
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ T sx[BK][BM + 1];
    __shared__ T sy[BK][BN + 1];
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    // one flat tile index (columns fastest) keeps every grid extent in range
    const int64_t ntn = (g.C + BN - 1) / BN, ntm = (g.R + BM - 1) / BM;
    const int64_t b = (int64_t)blockIdx.x / (ntn * ntm), rem = (int64_t)blockIdx.x - b * ntn * ntm;
    const int64_t r0 = (rem / ntn) * BM, c0 = (rem % ntn) * BN;
    const T *X = (const T *)g.X + b * g.bsx;
    const T *Y = (const T *)g.Y + b * g.bsy;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;
    for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int e = t + i * 256, rr = e / BK, kk = e % BK;
            int64_t gr = r0 + rr, gc = c0 + rr, gk = k0 + kk;
            sx[kk][rr] = (gr < g.R && gk < g.K) ? X[gr * g.ldx + gk] : T(0);
            sy[kk][rr] = (gc < g.C && gk < g.K) ? Y[gc * g.ldy + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sx[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) c[j] = sy[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * c[j];
        }
        __syncthreads();
    }
    T mx = 0;
    T *D = (T *)g.D + b * g.bsd;
    const T sxs = g.mxsx ? pow2neg<T>(exp_of_bits(*g.mxsx)) : T(1);
    int64_t rowlast = r0 + ty * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = r0 + ty * 4 + i;
        if (r >= g.R) continue;
        rowlast = r;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t c = c0 + tx * 4 + j;
            if (c < g.C) {
                const T v = acc[i][j] * sxs;
                D[r * g.ldd + c] = v;
                mx = mx > v ? mx : v;
            }
        }
    }
    bool any = r0 + ty * 4 < g.R;
    int64_t beta = g.beta_div_batch > 0 ? b / g.beta_div_batch
                   : g.beta_div_row > 0 ? (any ? rowlast : g.R - 1) / g.beta_div_row
                                        : 0;
    // rows ty*4..ty*4+3 of one thread may straddle items only if an item has
    // fewer than 4 rows; record per row in that case
    if (g.beta_div_row > 0 && g.beta_div_row < 4 && g.beta_div_batch <= 0) {
        for (int i = 0; i < 4; ++i) {
            int64_t r = r0 + ty * 4 + i;
            double m1 = 0;
            for (int j = 0; j < 4; ++j) {
                int64_t c = c0 + tx * 4 + j;
                if (r < g.R && c < g.C) m1 = fmax(m1, (double)acc[i][j]);
            }
            if (g.mxd && r < g.R && m1 > 0) atomicMax(g.mxd + r / g.beta_div_row, dbits(m1));
        }
        return;
    }
    record_max(g.mxd, beta, any, (double)mx);
}

void launch_simt_gemm(const GDesc &g, cudaStream_t st) {
    dim3 grid((unsigned)(((g.C + 63) / 64) * ((g.R + 63) / 64) * g.batch), 1, 1);
    if (g.xtype == E_F64) k_simt_gemm<double><<<grid, 256, 0, st>>>(g);
    else k_simt_gemm<float><<<grid, 256, 0, st>>>(g);
}

}  // namespace tn

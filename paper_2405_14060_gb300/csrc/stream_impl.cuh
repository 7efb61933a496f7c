// Streaming kernels for the HBM-bound absorptions of a contraction tree (a
// big tensor times a small one, which dominate a tree's read-write
// complexity, paper Sec. Benchmarks).  The big operand is read from HBM
// exactly once:
//
//   k_absorb       one thread per position r kept from the streamed operand X;
//                  it loads X[r, s] for every summed combination s into
//                  registers and writes Y[t, r] for every new combination t
//                  from the small operand W (read through L1).  Sum-product
//                  with power-of-two rescaling, or max-plus with the flat index
//                  of the maximiser (Eq. tropical).
//   k_absorb_sm    the sum-product form with W staged in shared memory, for
//                  many (summed x new) combinations per position.
//
// The reductions of two big tensors to a small one are in reduce_impl.cuh.
#include <cmath>

#pragma once
#include <algorithm>
#include <mutex>
#include <vector>

#include "dense_impl.cuh"
#include "devutil.cuh"
#include "stream.cuh"

namespace tn {

// Inner positions (the fastest dims, at most A_INNER entries) get their offsets
// from a table computed on the host when the node is planned (device memory,
// read through L1); each outer index is decoded once for its whole inner
// slice.  A position then costs one cached table load per operand plus its
// data accesses.
constexpr int A_INNER = 2048;

template <typename T, int NS, int NT, int SEMI>
__global__ void __launch_bounds__(256) k_absorb(const __grid_constant__ ADesc d) {
    constexpr int U = NS * NT <= 4 ? 8 : NS * NT <= 16 ? 4 : NS * NT <= 64 ? 2 : 1;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *ty = d.tab + nin, *tw = d.tab + 2 * nin;
    const int nod = d.nrd - d.nin_d;
    const int64_t beta = blockIdx.y;
    T mx = 0;
    T scale = T(1);
    // max-plus: the operands' recorded maxima are subtracted (max-normalised
    // inputs) and the output's maximum is recorded
    T offx = T(0), offw = T(0), mxq = -INFINITY;
    if (SEMI == SUM) {
        T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
        T sw = d.mxw ? pow2neg<T>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : T(1);
        scale = sx * sw;
    } else {
        offx = d.mxx ? okey_off<T>(d.mxx[beta * d.mxx_bs]) : T(0);
        offw = d.mxw ? okey_off<T>(d.mxw[beta * d.mxw_bs]) : T(0);
    }
    // tiles: (outer index, chunk of 256 U inner positions)
    const int nch = (nin + 256 * U - 1) / (256 * U);
    const int64_t ntile = d.nouter * nch;
    const int lnch = log2_if_pow2(nch);
    // With at least one outer index per block, block b takes outer indices
    // b, b + G, ... with all their chunks (the decode is reused across the
    // chunks, and blocks running together cover one band of the tensors);
    // otherwise the tiles are interleaved over the blocks.
    const bool by_outer = d.nouter >= (int64_t)gridDim.x;
    const int64_t nmine =
        by_outer ? ((d.nouter - blockIdx.x + gridDim.x - 1) / gridDim.x) * nch
                 : (ntile > blockIdx.x ? (ntile - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);
    int64_t cur_o = -1, bx = 0, by = 0, bw = 0;
    for (int64_t k = 0; k < nmine; ++k) {
        int64_t crem, o;
        if (by_outer) {
            const int64_t ko = div_tile(k, nch, lnch, crem);
            o = (int64_t)blockIdx.x + ko * gridDim.x;
        } else {
            o = div_tile((int64_t)blockIdx.x + k * gridDim.x, nch, lnch, crem);
        }
        const int c = (int)crem;
        if (o != cur_o) {
            cur_o = o;
            bx = beta * d.bsx;
            by = beta * d.bsy;
            bw = beta * d.bsw;
            if (d.pow2r) {
                const int64_t r0 = o * nin;
                for (int k = 0; k < nod; ++k) {
                    int64_t dg = (r0 >> d.rsh[k]) & (int64_t)(d.rsz[k] - 1);
                    bx += dg * d.rsx[k];
                    by += dg * d.rsy[k];
                    bw += dg * d.rsw[k];
                }
            } else {
                int64_t r = o;
                for (int k = nod - 1; k >= 0; --k) {
                    int64_t dg = r % d.rsz[k];
                    r /= d.rsz[k];
                    bx += dg * d.rsx[k];
                    by += dg * d.rsy[k];
                    bw += dg * d.rsw[k];
                }
            }
        }
        const T *Xb = (const T *)d.X + bx;
        const T *Wb = (const T *)d.W + bw;
        T *Yb = (T *)d.Y + by;
        {
            const int j0 = c * 256 * U + threadIdx.x;
            T x[U][NS];
            int oy[U], ow[U];
            bool on[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int j = j0 + u * 256;
                on[u] = j < nin;
                int jj = on[u] ? j : 0;
                int ox = __ldg(tx + jj);
                oy[u] = __ldg(ty + jj);
                ow[u] = __ldg(tw + jj);
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    x[u][s] = (on[u] && (NS == 1 || s < d.ns)) ? Xb[ox + d.xoff[s]] - offx : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!on[u]) continue;
                const T *W = Wb + ow[u];
                T *Y = Yb + oy[u];
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    if (NT > 1 && t >= d.nt) break;
                    if (SEMI == SUM) {
                        T acc = 0;
#pragma unroll
                        for (int s = 0; s < NS; ++s)
                            if (NS == 1 || s < d.ns) acc += x[u][s] * __ldg(W + d.wso[s] + d.wto[t]);
                        Y[d.yoff[t]] = acc * scale;
                        mx = mx > acc ? mx : acc;
                    } else {
                        T best = -INFINITY;
                        int32_t bk = 0;
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            if (NS > 1 && s >= d.ns) break;
                            T v = x[u][s] + (__ldg(W + d.wso[s] + d.wto[t]) - offw);
                            if (v > best) { best = v; bk = s; }
                        }
                        Y[d.yoff[t]] = best;
                        mxq = mxq > best ? mxq : best;
                        if (d.argmax) d.argmax[by + oy[u] + d.yoff[t]] = bk;
                    }
                }
            }
        }
    }
    if (SEMI == SUM && d.mxy) block_max_atomic(d.mxy + beta, (double)mx * (double)scale);
    if (SEMI == MAXPLUS) record_max_key(d.mxy, beta, true, (double)mxq);
}

// Sum-product absorb with many (summed x new) combinations per position.
// The small operand W is staged once per block in shared memory as dense
// [shared combination][s][t] blocks (t fastest, zero-padded to NS x NT, one
// padding quad between blocks to spread banks), so the inner loop is
// register-blocked: each thread keeps its position's NS values of X in
// registers and reads W a vector of t values at a time (VW FMAs per shared
// load) instead of one global load per multiply-add.
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int W = 4;
};
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int W = 2;
};

template <typename T, int NS, int NT>
__host__ __device__ constexpr int absorb_blk() {
    return NS * NT + 16 / (int)sizeof(T);
}

template <typename T, int NS, int NT>
__global__ void __launch_bounds__(256) k_absorb_sm(const __grid_constant__ ADesc d) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *smW = (T *)smraw;
    constexpr int BLK = absorb_blk<T, NS, NT>();
    constexpr int VW = NT < Vec<T>::W ? NT : Vec<T>::W;
    constexpr int U = NS * NT <= 64 ? 2 : 1;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *ty = d.tab + nin, *tc = d.tab + 3 * nin, *wsh = d.tab + 4 * nin;
    const int nod = d.nrd - d.nin_d;
    const int64_t beta = blockIdx.y;
    {
        const T *Wg = (const T *)d.W + beta * d.bsw;
        const int tot = d.nsh * NS * NT;
        for (int i = threadIdx.x; i < tot; i += 256) {
            int c = i / (NS * NT), st = i - c * (NS * NT);
            int si = st / NT, ti = st - si * NT;
            T v = T(0);
            if (si < d.ns && ti < d.nt) v = __ldg(Wg + wsh[c] + d.wso[si] + d.wto[ti]);
            smW[c * BLK + st] = v;
        }
    }
    __syncthreads();
    T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    T sw = d.mxw ? pow2neg<T>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : T(1);
    const T scale = sx * sw;
    T mx = 0;
    const int nch = (nin + 256 * U - 1) / (256 * U);
    const int64_t ntile = d.nouter * nch;
    const int lnch = log2_if_pow2(nch);
    // With at least one outer index per block, block b takes outer indices
    // b, b + G, ... with all their chunks (the decode is reused across the
    // chunks, and blocks running together cover one band of the tensors);
    // otherwise the tiles are interleaved over the blocks.
    const bool by_outer = d.nouter >= (int64_t)gridDim.x;
    const int64_t nmine =
        by_outer ? ((d.nouter - blockIdx.x + gridDim.x - 1) / gridDim.x) * nch
                 : (ntile > blockIdx.x ? (ntile - blockIdx.x + gridDim.x - 1) / gridDim.x : 0);
    int64_t cur_o = -1, bx = 0, by = 0;
    int cb = 0;
    for (int64_t k = 0; k < nmine; ++k) {
        int64_t crem, o;
        if (by_outer) {
            const int64_t ko = div_tile(k, nch, lnch, crem);
            o = (int64_t)blockIdx.x + ko * gridDim.x;
        } else {
            o = div_tile((int64_t)blockIdx.x + k * gridDim.x, nch, lnch, crem);
        }
        const int c = (int)crem;
        if (o != cur_o) {
            cur_o = o;
            bx = beta * d.bsx;
            by = beta * d.bsy;
            cb = 0;
            if (d.pow2r) {
                const int64_t r0 = o * nin;
                for (int k = 0; k < nod; ++k) {
                    int64_t dg = (r0 >> d.rsh[k]) & (int64_t)(d.rsz[k] - 1);
                    bx += dg * d.rsx[k];
                    by += dg * d.rsy[k];
                    cb += (int)dg * d.rshc[k];
                }
            } else {
                int64_t r = o;
                for (int k = nod - 1; k >= 0; --k) {
                    int64_t dg = r % d.rsz[k];
                    r /= d.rsz[k];
                    bx += dg * d.rsx[k];
                    by += dg * d.rsy[k];
                    cb += (int)dg * d.rshc[k];
                }
            }
        }
        const T *Xb = (const T *)d.X + bx;
        T *Yb = (T *)d.Y + by;
        {
            const int j0 = c * 256 * U + threadIdx.x;
            T x[U][NS];
            int oy[U], oc[U];
            bool on[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int j = j0 + u * 256;
                on[u] = j < nin;
                int jj = on[u] ? j : 0;
                int ox = __ldg(tx + jj);
                oy[u] = __ldg(ty + jj);
                oc[u] = (cb + __ldg(tc + jj)) * BLK;
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    x[u][s] = (on[u] && s < d.ns) ? Xb[ox + d.xoff[s]] : T(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!on[u]) continue;
                const T *w = smW + oc[u];
                T *Y = Yb + oy[u];
#pragma unroll
                for (int t0 = 0; t0 < NT; t0 += VW) {
                    if (t0 >= d.nt) break;
                    T acc[VW];
#pragma unroll
                    for (int v = 0; v < VW; ++v) acc[v] = 0;
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        if (VW == Vec<T>::W) {
                            typename Vec<T>::V wv = *(const typename Vec<T>::V *)(w + s * NT + t0);
                            const T *wp = (const T *)&wv;
#pragma unroll
                            for (int v = 0; v < VW; ++v) acc[v] += x[u][s] * wp[v];
                        } else {
#pragma unroll
                            for (int v = 0; v < VW; ++v) acc[v] += x[u][s] * w[s * NT + t0 + v];
                        }
                    }
#pragma unroll
                    for (int v = 0; v < VW; ++v) {
                        if (t0 + v < d.nt) {
                            Y[d.yoff[t0 + v]] = acc[v] * scale;
                            mx = mx > acc[v] ? mx : acc[v];
                        }
                    }
                }
            }
        }
    }
    if (d.mxy) block_max_atomic(d.mxy + beta, (double)mx * (double)scale);
}

// Vector form of the sum-product absorb (FP32 data): where the fastest kept
// dimension is contiguous in X and Y and absent from W, a thread takes four
// consecutive positions, loads X 16 bytes per summed combination, stores Y
// 16 bytes per new combination, and reads each W value (shared memory,
// [shared combination][s][t]) once for four multiply-adds.  New combinations
// go in groups of 8 (X re-read per group, from L1).
static __global__ void __launch_bounds__(256) k_absorb_v4(const __grid_constant__ ADesc d) {
    extern __shared__ __align__(16) float smw4[];
    const int ns = d.ns, nt = d.nt, nst = ns * nt;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *ty = d.tab + nin, *tc = d.tab + 3 * nin, *wsh = d.tab + 4 * nin;
    const int nod = d.nrd - d.nin_d;
    const int64_t beta = blockIdx.y;
    {
        const float *Wg = (const float *)d.W + beta * d.bsw;
        for (int i = threadIdx.x; i < d.nsh * nst; i += 256) {
            const int c = i / nst, r = i - c * nst, si = r / nt, ti = r - si * nt;
            smw4[i] = __ldg(Wg + wsh[c] + d.wso[si] + d.wto[ti]);
        }
    }
    __syncthreads();
    const float sx = d.mxx ? pow2neg<float>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : 1.f;
    const float sw = d.mxw ? pow2neg<float>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : 1.f;
    const float scale = sx * sw;
    float mx = 0.f;
    const int nq = nin >> 2;
    const int nch = (nq + 255) / 256;
    const int lnch = log2_if_pow2(nch);
    const int64_t ntile = d.nouter * nch;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        int64_t crem;
        const int64_t o = div_tile(tile, nch, lnch, crem);
        const int j = (int)crem * 256 + threadIdx.x;   // quad of inner positions
        if (j >= nq) continue;
        int64_t bx = beta * d.bsx, by = beta * d.bsy;
        int cb = 0;
        if (d.pow2r) {
            const int64_t r0 = o * nin;
            for (int k = 0; k < nod; ++k) {
                const int64_t dg = (r0 >> d.rsh[k]) & (int64_t)(d.rsz[k] - 1);
                bx += dg * d.rsx[k];
                by += dg * d.rsy[k];
                cb += (int)dg * d.rshc[k];
            }
        } else {
            int64_t r = o;
            for (int k = nod - 1; k >= 0; --k) {
                const int64_t dg = r % d.rsz[k];
                r /= d.rsz[k];
                bx += dg * d.rsx[k];
                by += dg * d.rsy[k];
                cb += (int)dg * d.rshc[k];
            }
        }
        const int p = 4 * j;
        const float *Xq = (const float *)d.X + bx + __ldg(tx + p);
        float *Yq = (float *)d.Y + by + __ldg(ty + p);
        const float *wq = smw4 + (cb + __ldg(tc + p)) * nst;
        for (int t0 = 0; t0 < nt; t0 += 8) {
            float4 acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int si = 0; si < ns; ++si) {
                const float4 x = __ldg((const float4 *)(Xq + d.xoff[si]));
                const float *w = wq + si * nt + t0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (t0 + u < nt) {
                        const float wv = w[u];
                        acc[u].x += x.x * wv;
                        acc[u].y += x.y * wv;
                        acc[u].z += x.z * wv;
                        acc[u].w += x.w * wv;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (t0 + u < nt) {
                    const float4 a = acc[u];
                    *(float4 *)(Yq + d.yoff[t0 + u]) =
                        make_float4(a.x * scale, a.y * scale, a.z * scale, a.w * scale);
                    mx = fmaxf(mx, fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)));
                }
            }
        }
    }
    if (d.mxy) block_max_atomic(d.mxy + beta, (double)mx * (double)scale);
}

// Can the absorb run as k_absorb_v4 (host)?
static bool absorb_v4_form(const ADesc &d) {
    const int L = d.nrd - 1;
    if (L < 0 || d.nin_d < 1) return false;
    if (d.rsx[L] != 1 || d.rsy[L] != 1 || d.rsw[L] != 0 || d.rshc[L] != 0 || d.rsz[L] % 4 ||
        d.nin % 4)
        return false;
    if (((uintptr_t)d.X & 15) || ((uintptr_t)d.Y & 15) || d.bsx % 4 || d.bsy % 4) return false;
    for (int k = 0; k < L; ++k)
        if (d.rsx[k] % 4 || d.rsy[k] % 4) return false;
    for (int i = 0; i < d.ns; ++i)
        if (d.xoff[i] % 4) return false;
    for (int i = 0; i < d.nt; ++i)
        if (d.yoff[i] % 4) return false;
    // more combinations than 128: the register-blocked kernel measured faster
    // (24 x 24 grid: 32 x 8 absorbs 3.0-3.5 TB/s there against 2.4-2.6 here)
    return d.ns * d.nt <= 128 && (size_t)d.nsh * d.ns * d.nt * 4 <= 32768;
}

template <typename T, int NS, int NT>
static void absorb_go(const ADesc &d, int semiring, cudaStream_t st) {
    constexpr int BLK = absorb_blk<T, NS, NT>();
    const size_t smem = (size_t)d.nsh * BLK * sizeof(T);
    if constexpr (NS * NT >= 16) {
        if (semiring == SUM && smem <= 32768) {
            // a few resident blocks per SM, each stages W once
            constexpr int U = NS * NT <= 64 ? 2 : 1;
            int64_t ntile = d.nouter * ((d.nin + 256 * U - 1) / (256 * U));
            int64_t cap = std::max<int64_t>(1, (152LL * (d.bps > 0 ? d.bps : 4)) / std::max(1, d.nbeta));
            dim3 grid((unsigned)std::max<int64_t>(1, std::min(ntile, cap)), (unsigned)d.nbeta, 1);
            k_absorb_sm<T, NS, NT><<<grid, 256, smem, st>>>(d);
            return;
        }
    }
    constexpr int U = NS * NT <= 4 ? 8 : NS * NT <= 16 ? 4 : NS * NT <= 64 ? 2 : 1;
    int64_t ntile = d.nouter * ((d.nin + 256 * U - 1) / (256 * U));
    int64_t cap = std::max<int64_t>(1, (152LL * (d.bps > 0 ? 4 * d.bps : 16)) / std::max(1, d.nbeta));
    dim3 grid((unsigned)std::max<int64_t>(1, std::min(ntile, cap)), (unsigned)d.nbeta, 1);
    if (semiring == SUM) k_absorb<T, NS, NT, SUM><<<grid, 256, 0, st>>>(d);
    else k_absorb<T, NS, NT, MAXPLUS><<<grid, 256, 0, st>>>(d);
}

// Exact instantiations for every (ns, nt) up to 32; a combination count that
// is not a power of two runs on the next power of two with padded offsets.
template <typename T, int NS>
static void absorb_nt(const ADesc &d, int nt, int semiring, cudaStream_t st) {
    switch (nt) {
        case 1: absorb_go<T, NS, 1>(d, semiring, st); break;
        case 2: absorb_go<T, NS, 2>(d, semiring, st); break;
        case 4: absorb_go<T, NS, 4>(d, semiring, st); break;
        case 8: absorb_go<T, NS, 8>(d, semiring, st); break;
        case 16: absorb_go<T, NS, (NS <= 16 ? 16 : 8)>(d, semiring, st); break;
        default: absorb_go<T, NS, (NS <= 8 ? 32 : 8)>(d, semiring, st); break;
    }
}

static int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Launch modes of the dense absorb (host): 16-byte copies and stores where
// every aligned quad of consecutive entries is contiguous and 16-byte aligned.
static DenseModes absorb_dense_modes(const ADesc &d) {
    DenseModes m{0, 0};
    const int L = d.nrd - 1;   // the fastest position dim
    auto aligned = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    auto strides4 = [&](const int64_t *st, int skip) {
        for (int k = 0; k < d.nrd; ++k)
            if (k != skip && st[k] % 4) return false;
        return true;
    };
    auto offs4 = [](const int32_t *o, int n) {
        for (int i = 0; i < n; ++i)
            if (o[i] % 4) return false;
        return true;
    };
    auto quads = [](const int32_t *o, int n) {
        if (n % 4) return false;
        for (int i = 0; i < n; ++i)
            if (o[i] != o[i & ~3] + (i & 3)) return false;
        return true;
    };
    const bool pos4 = d.nin % 4 == 0 && d.rsz[L] % 4 == 0;
    if (aligned(d.X) && d.bsx % 4 == 0) {
        if (pos4 && d.rsx[L] == 1 && strides4(d.rsx, L) && offs4(d.xoff, d.ns)) m.xm = 1;
        else if (strides4(d.rsx, -1) && quads(d.xoff, d.ns) && offs4(d.xoff, d.ns)) m.xm = 2;
    }
    if (aligned(d.Y) && d.bsy % 4 == 0) {
        if (pos4 && d.rsy[L] == 1 && strides4(d.rsy, L) && offs4(d.yoff, d.nt)) m.ym = 1;
        else if (strides4(d.rsy, -1) && quads(d.yoff, d.nt) && offs4(d.yoff, d.nt)) m.ym = 2;
    }
    // otherwise the planned chunk tables, where the layout allows them
    if (m.xm == 0 && d.cx) m.xm = 3;
    if (m.ym == 0 && d.cy) m.ym = 3;
    return m;
}

template <typename T, int XM>
static void absorb_dense_go(const ADesc &d, int ym, cudaStream_t st) {
    constexpr size_t smem = absorb_dense_smem<T, XM>();
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_absorb_dense<T, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    });
    const int bps = (int)std::max<size_t>(1, (227 * 1024) / (smem + 1024));
    const int64_t ntile = d.nouter * ((d.nin + AD_P - 1) / AD_P);
    const int64_t cap = std::max<int64_t>(1, (152LL * bps) / std::max(1, d.nbeta));
    dim3 grid((unsigned)std::max<int64_t>(1, std::min(ntile, cap)), (unsigned)d.nbeta, 1);
    k_absorb_dense<T, XM><<<grid, AD_T, smem, st>>>(d, ym);
}

// Does the absorb run as k_absorb_dense (more than 256 combinations after
// rounding to powers of two; sum-product with W holding no position label)?
static bool absorb_dense_form(const ADesc &d) {
    return pow2ceil(d.ns) * pow2ceil(d.nt) > 256;
}

#ifdef TN_STREAM_HOST_DEFS
bool absorb_dense_form_host(const ADesc &d) { return absorb_dense_form(d); }
void absorb_dense_describe(const ADesc &d, int &xm, int &ym) {
    xm = ym = -1;
    if (!absorb_dense_form(d)) return;
    const DenseModes m = absorb_dense_modes(d);
    xm = m.xm;
    ym = m.ym;
}
#endif

template <typename T>
void launch_absorb(const ADesc &d0, int semiring, cudaStream_t st) {
    if (d0.nr * d0.nbeta == 0) return;
    ADesc d = d0;
    if (absorb_dense_form(d)) {
        if (semiring != SUM || d.nsh != 1 || d.ns > 32 || d.nt > 32) return;
        const DenseModes m = absorb_dense_modes(d);
        if (m.xm == 1) absorb_dense_go<T, 1>(d, m.ym, st);
        else if (m.xm == 2) absorb_dense_go<T, 2>(d, m.ym, st);
        else if (m.xm == 3) absorb_dense_go<T, 3>(d, m.ym, st);
        else absorb_dense_go<T, 0>(d, m.ym, st);
        return;
    }
    // FP32 sum-product with a contiguous fastest kept dimension: the vector
    // form
    if constexpr (sizeof(T) == 4) {
        if (semiring == SUM && absorb_v4_form(d)) {
            const int64_t ntile = d.nouter * ((d.nin / 4 + 255) / 256);
            const int64_t cap = std::max<int64_t>(
                1, (152LL * (d.bps > 0 ? 2 * d.bps : 8)) / std::max(1, d.nbeta));
            dim3 grid((unsigned)std::max<int64_t>(1, std::min(ntile, cap)), (unsigned)d.nbeta, 1);
            k_absorb_v4<<<grid, 256, (size_t)d.nsh * d.ns * d.nt * 4, st>>>(d);
            return;
        }
    }
    // the kernel runs on the next powers of two; the extra combinations are
    // skipped by warp-uniform guards
    int ns = pow2ceil(d.ns), nt = pow2ceil(d.nt);
    if (ns > 32 || nt > 32 || ns * nt > 256) return;
    (void)ns;
    switch (ns) {
        case 1: absorb_nt<T, 1>(d, nt, semiring, st); break;
        case 2: absorb_nt<T, 2>(d, nt, semiring, st); break;
        case 4: absorb_nt<T, 4>(d, nt, semiring, st); break;
        case 8: absorb_nt<T, 8>(d, nt, semiring, st); break;
        case 16: absorb_nt<T, 16>(d, nt, semiring, st); break;
        default: absorb_nt<T, 32>(d, nt, semiring, st); break;
    }
}

}  // namespace tn

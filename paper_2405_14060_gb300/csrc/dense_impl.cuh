// Dense streaming contractions for nodes with many summed x new combinations
// (more than the register-blocked absorb and reduce kernels take, up to
// 32 x 32): a big tensor against a small dense block, the shape that binary
// labels give when five labels are summed and five are new, and the
// adjoint steps of such nodes (Thm. "Tensor network differentiation",
// Eq. einback).  Both read every entry of the big operands from HBM once.
//
//   k_absorb_dense   Y[t, r] = sum_s X[r, s] W[s, t]: W staged once per block
//                    in shared memory as [s][t]; tiles of 128 positions r of X
//                    staged by asynchronous copies two tiles ahead (as [s][p]
//                    when positions are contiguous in X, as [p][s] when the
//                    summed combinations are); each of 128 threads owns 8
//                    positions x 4 new combinations and reads 16-byte vectors
//                    of both (three shared loads per 32 multiply-adds).
//   k_reduce_dense   O[g, s, t] = sum_m X[g, m, s] Z[g, m, t]: tiles of 64
//                    positions of both operands staged as [p][s | t]; four
//                    thread groups take a quarter of each tile's positions,
//                    each thread 4 x 4 outputs of the 32 x 32 block; per-block
//                    partials summed by the group's last block in a fixed order
//                    (deterministic).
#pragma once
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "devutil.cuh"
#include "stream.cuh"

namespace tn {

// Group offsets of a reduce descriptor's group index gi in X, Z and O.
__device__ __forceinline__ void group_offsets(const RDesc &d, int64_t gi, int64_t &ox,
                                              int64_t &oz, int64_t &oo) {
    for (int i = d.ngd - 1; i >= 0; --i) {
        int64_t dg = gi % d.gsz[i];
        gi /= d.gsz[i];
        ox += dg * d.gsx[i];
        oz += dg * d.gsz2[i];
        oo += dg * d.gso[i];
    }
}

// Outer decode of the summed positions: operand offsets of outer index o.
__device__ __forceinline__ void reduce_outer(const RDesc &d, int64_t o, int nod, int64_t &cbx,
                                             int64_t &cbz) {
    if (d.pow2m) {
        const int64_t r0 = o * d.nin;
        for (int q = 0; q < nod; ++q) {
            int64_t dg = (r0 >> d.msh[q]) & (int64_t)(d.msz[q] - 1);
            cbx += dg * d.msx[q];
            cbz += dg * d.msz2[q];
        }
    } else {
        int64_t r = o;
        for (int q = nod - 1; q >= 0; --q) {
            int64_t dg = r % d.msz[q];
            r /= d.msz[q];
            cbx += dg * d.msx[q];
            cbz += dg * d.msz2[q];
        }
    }
}

// Four consecutive entries as 16-byte vectors (one float4, two double2).
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 a = *(const float4 *)p;
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = *(const double2 *)p, b = *(const double2 *)(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d) {
    *(float4 *)p = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double *p, double a, double b, double c, double d) {
    *(double2 *)p = make_double2(a, b);
    *(double2 *)(p + 2) = make_double2(c, d);
}
// Asynchronous copy of four consecutive entries (16 bytes per instruction),
// zeros instead when !ok.
template <typename T>
__device__ __forceinline__ void cp_async4(uint32_t s, const T *g, bool ok) {
#pragma unroll
    for (int h = 0; h < (int)sizeof(T) / 4; ++h)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s + 16 * h),
                     "l"(g + h * (16 / (int)sizeof(T))), "r"(ok ? 16 : 0)
                     : "memory");
}
// One entry, zeros instead when !ok.
template <typename T>
__device__ __forceinline__ void cp_async1(uint32_t s, const T *g, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(s), "l"(g),
                 "n"(sizeof(T)), "r"(ok ? (int)sizeof(T) : 0)
                 : "memory");
}

// Launch modes of the dense absorb, chosen on the host from the descriptor:
// X: 0 one entry per copy into [s][p], 1 four positions per copy into
// [s][p], 2 four summed combinations per copy into [p][s], 3 the tile's
// 16-byte chunks in memory order (planned table), scattered into [s][p];
// Y: 0 one entry per store, 1 four positions per store, 2 four new
// combinations per store, 3 the tile's chunks through shared memory.
struct DenseModes {
    int xm, ym;
};

constexpr int AD_P = 128;   // positions per tile
constexpr int AD_T = 128;   // threads: 8 positions x 4 new combinations each
constexpr int AD_S = 3;     // tile buffers

template <typename T>
__host__ __device__ constexpr int ad_pad() {
    return 16 / (int)sizeof(T);
}
// Entries of one tile buffer for X mode XM: [s][p] (0, 1), [p][s] (2), the
// tile's chunks in memory order (3).
template <typename T, int XM>
__host__ __device__ constexpr int ad_buf() {
    return XM == 3 ? 32 * AD_P : XM == 2 ? AD_P * (32 + ad_pad<T>()) : 32 * (AD_P + ad_pad<T>());
}
template <typename T, int XM>
__host__ __device__ constexpr size_t absorb_dense_smem() {
    // W [32][32 + pad], tile buffers, and in chunk mode the [s][p] tile the
    // chunks are scattered into
    return ((size_t)32 * (32 + ad_pad<T>()) + (size_t)AD_S * ad_buf<T, XM>() +
            (XM == 3 ? (size_t)32 * (AD_P + ad_pad<T>()) : 0)) *
           sizeof(T);
}

// Outer decode of position tile o (outer index): operand bases.
__device__ __forceinline__ void absorb_outer(const ADesc &d, int64_t o, int nod, int64_t &bx,
                                             int64_t &by) {
    if (d.pow2r) {
        const int64_t r0 = o * d.nin;
        for (int k = 0; k < nod; ++k) {
            const int64_t dg = (r0 >> d.rsh[k]) & (int64_t)(d.rsz[k] - 1);
            bx += dg * d.rsx[k];
            by += dg * d.rsy[k];
        }
    } else {
        int64_t r = o;
        for (int k = nod - 1; k >= 0; --k) {
            const int64_t dg = r % d.rsz[k];
            r /= d.rsz[k];
            bx += dg * d.rsx[k];
            by += dg * d.rsy[k];
        }
    }
}

// Four entries of a tile buffer scattered to (or gathered from) the 16-bit
// shared-memory slots packed in w.
template <typename T>
__device__ __forceinline__ void scatter4(T *dst, uint2 w, const T (&v)[4]) {
    dst[w.x & 0xffffu] = v[0];
    dst[w.x >> 16] = v[1];
    dst[w.y & 0xffffu] = v[2];
    dst[w.y >> 16] = v[3];
}

// ym: 0 one entry per store, 1 four positions per store, 2 four new
// combinations per store (all from registers), 3 through shared memory as
// the tile's chunks in memory order (chunk table at d.cyo).
template <typename T, int XM>
__global__ void __launch_bounds__(AD_T) k_absorb_dense(const __grid_constant__ ADesc d, int ym) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int PAD = ad_pad<T>();
    constexpr int WR = 32 + PAD;                       // W row: [s][t]
    constexpr int RS = AD_P + PAD;                     // [s][p] / [t][p] row
    constexpr int RX = XM == 2 ? 32 + PAD : RS;        // row of the tile buffers
    constexpr int TB = ad_buf<T, XM>();
    T *Ws = (T *)smraw;
    T *Xs = Ws + 32 * WR;
    T *Xc = Xs + AD_S * TB;                            // chunk mode: [s][p]
    const int tid = threadIdx.x;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *ty = d.tab + nin;
    const int nod = d.nrd - d.nin_d;
    const int64_t beta = blockIdx.y;
    const int ns4 = (d.ns + 3) & ~3;
    const int nqx = d.ns * (AD_P / 4), nqy = d.nt * (AD_P / 4);
    {
        const T *Wg = (const T *)d.W + beta * d.bsw;
        for (int i = tid; i < 32 * 32; i += AD_T) {
            const int s = i >> 5, t = i & 31;
            Ws[s * WR + t] = (s < d.ns && t < d.nt) ? __ldg(Wg + d.wso[s] + d.wto[t]) : T(0);
        }
    }
    const T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    const T sw = d.mxw ? pow2neg<T>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : T(1);
    const T scale = sx * sw;
    const int nch = (nin + AD_P - 1) / AD_P;
    const int64_t ntile = d.nouter * nch;
    const int lnch = log2_if_pow2(nch);
    const int64_t mine =
        ntile > blockIdx.x ? (ntile - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const T *X = (const T *)d.X + beta * d.bsx;
    T *Y = (T *)d.Y + beta * d.bsy;
    const uint32_t xs0 = (uint32_t)__cvta_generic_to_shared(Xs);
    // X chunk mode: this thread's chunks q = tid + AD_T r are the same in
    // every tile, so their offsets and slots stay in registers
    constexpr int NQ = 32 * (AD_P / 4) / AD_T;
    int32_t xrel[NQ];
    uint2 xsl[NQ];
#pragma unroll
    for (int r = 0; r < NQ; ++r) {
        const int q = tid + AD_T * r;
        xrel[r] = 0;
        xsl[r] = make_uint2(0u, 0u);
        if (XM == 3 && q < nqx) {
            xrel[r] = __ldg(d.tab + d.cxo + q);
            xsl[r] = __ldg((const uint2 *)(d.tab + d.cxo + nqx) + q);
        }
    }
    // copies of this block's k-th tile into buffer b (an empty group past the end)
    auto issue = [&](int64_t k, int b) {
        if (k < mine) {
            int64_t crem;
            const int64_t o = div_tile((int64_t)blockIdx.x + k * gridDim.x, nch, lnch, crem);
            int64_t bx = 0, by = 0;
            absorb_outer(d, o, nod, bx, by);
            const int j0 = (int)crem * AD_P;
            const T *Xo = X + bx;
            const uint32_t sb = xs0 + (uint32_t)(b * TB * sizeof(T));
            if (XM == 3) {
                const T *Xt = Xo + __ldg(tx + j0);
#pragma unroll
                for (int r = 0; r < NQ; ++r) {
                    const int q = tid + AD_T * r;
                    if (q < nqx)
                        cp_async4<T>(sb + (uint32_t)(4 * q * sizeof(T)), Xt + xrel[r], true);
                }
            } else if (XM == 1) {
                // 32 rows x 32 quads of positions
                for (int e = tid; e < 32 * (AD_P / 4); e += AD_T) {
                    const int s = e / (AD_P / 4), p = (e % (AD_P / 4)) * 4;
                    const int j = j0 + p;
                    const bool ok = s < d.ns && j < nin;
                    cp_async4<T>(sb + (uint32_t)((s * RX + p) * sizeof(T)),
                                 ok ? Xo + __ldg(tx + j) + d.xoff[s] : Xo, ok);
                }
            } else if (XM == 2) {
                // AD_P rows x 8 quads of summed combinations
                for (int e = tid; e < AD_P * 8; e += AD_T) {
                    const int p = e >> 3, s = (e & 7) * 4;
                    const int j = j0 + p;
                    const bool ok = s < d.ns && j < nin;
                    cp_async4<T>(sb + (uint32_t)((p * RX + s) * sizeof(T)),
                                 ok ? Xo + __ldg(tx + j) + d.xoff[s] : Xo, ok);
                }
            } else {
                for (int e = tid; e < 32 * AD_P; e += AD_T) {
                    const int s = e / AD_P, p = e % AD_P;
                    const int j = j0 + p;
                    const bool ok = s < d.ns && j < nin;
                    cp_async1<T>(sb + (uint32_t)((s * RX + p) * sizeof(T)),
                                 ok ? Xo + __ldg(tx + j) + d.xoff[s] : Xo, ok);
                }
            }
        }
        cp_async_commit();
    };
    const int pg = tid >> 3, tg = tid & 7;   // positions 8 pg + i, new combinations 4 tg + j
    T mx = 0;
    issue(0, 0);
    issue(1, 1);
    int b = 0;
    for (int64_t k = 0; k < mine; ++k) {
        cp_async_wait<1>();
        // tile k landed everywhere; every thread is done with tile k - 1
        __syncthreads();
        issue(k + 2, b == 0 ? 2 : b - 1);
        T *tb = Xs + b * TB;
        const T *xb = tb;
        if (XM == 3) {
#pragma unroll
            for (int r = 0; r < NQ; ++r) {
                const int q = tid + AD_T * r;
                if (q < nqx) {
                    T v[4];
                    ld4(tb + 4 * q, v);
                    scatter4(Xc, xsl[r], v);
                }
            }
            __syncthreads();
            xb = Xc;
        }
        T acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        if (XM == 2) {
            for (int s = 0; s < ns4; s += 4) {
                T xv[8][4], wv[4][4];
#pragma unroll
                for (int i = 0; i < 8; ++i) ld4(xb + (8 * pg + i) * RX + s, xv[i]);
#pragma unroll
                for (int q = 0; q < 4; ++q) ld4(Ws + (s + q) * WR + 4 * tg, wv[q]);
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] += xv[i][q] * wv[q][j];
            }
        } else {
            // chunk mode fills only the rows s < ns
            const int send = XM == 3 ? d.ns : ns4;
            for (int s = 0; s < send; ++s) {
                T xv[8], wv[4];
                ld4(xb + s * RS + 8 * pg, *(T(*)[4])xv);
                ld4(xb + s * RS + 8 * pg + 4, *(T(*)[4])(xv + 4));
                ld4(Ws + s * WR + 4 * tg, wv);
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += xv[i] * wv[j];
            }
        }
        int64_t crem;
        const int64_t o = div_tile((int64_t)blockIdx.x + k * gridDim.x, nch, lnch, crem);
        int64_t bx = 0, by = 0;
        absorb_outer(d, o, nod, bx, by);
        T *Yo = Y + by;
        const int j0 = (int)crem * AD_P + 8 * pg;
        const int t0 = 4 * tg;
        if (ym == 3) {
            // [t][p] in shared memory, then the tile's chunks in memory order
            T *ys = XM == 3 ? Xc : tb;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (t0 + j >= d.nt) break;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    st4(ys + (t0 + j) * RS + 8 * pg + 4 * h, acc[4 * h][j] * scale,
                        acc[4 * h + 1][j] * scale, acc[4 * h + 2][j] * scale,
                        acc[4 * h + 3][j] * scale);
#pragma unroll
                for (int i = 0; i < 8; ++i) mx = mx > acc[i][j] ? mx : acc[i][j];
            }
            __syncthreads();
            T *Yt = Yo + __ldg(ty + (int)crem * AD_P);
            const int32_t *cry = d.tab + d.cyo;
            const uint2 *csy = (const uint2 *)(d.tab + d.cyo + nqy);
            for (int q = tid; q < nqy; q += AD_T) {
                const uint2 w = __ldg(csy + q);
                st4(Yt + __ldg(cry + q), ys[w.x & 0xffffu], ys[w.x >> 16], ys[w.y & 0xffffu],
                    ys[w.y >> 16]);
            }
        } else if (ym == 1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jq = j0 + 4 * h;   // a quad of positions: all valid or none
                if (jq >= nin) continue;
                const int oy = __ldg(ty + jq);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (t0 + j >= d.nt) break;
                    st4(Yo + oy + d.yoff[t0 + j], acc[4 * h][j] * scale,
                        acc[4 * h + 1][j] * scale, acc[4 * h + 2][j] * scale,
                        acc[4 * h + 3][j] * scale);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        mx = mx > acc[4 * h + i][j] ? mx : acc[4 * h + i][j];
                }
            }
        } else if (ym == 2) {
            if (t0 < d.nt) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (j0 + i >= nin) break;
                    st4(Yo + __ldg(ty + j0 + i) + d.yoff[t0], acc[i][0] * scale,
                        acc[i][1] * scale, acc[i][2] * scale, acc[i][3] * scale);
#pragma unroll
                    for (int j = 0; j < 4; ++j) mx = mx > acc[i][j] ? mx : acc[i][j];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (j0 + i >= nin) break;
                const int oy = __ldg(ty + j0 + i);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (t0 + j >= d.nt) break;
                    Yo[oy + d.yoff[t0 + j]] = acc[i][j] * scale;
                    mx = mx > acc[i][j] ? mx : acc[i][j];
                }
            }
        }
        b = b == 2 ? 0 : b + 1;
    }
    cp_async_wait<0>();
    if (d.mxy) block_max_atomic(d.mxy + beta, (double)mx * (double)scale);
}

constexpr int RD_P = 64;    // positions per tile
constexpr int RD_S = 3;     // tile buffers

// Per tile buffer: the [64 rows: X s, then Z t][RD_P + pad] tile and, for
// each operand copied as planned chunks (chunk mode), a staging area of its
// 32 x RD_P entries in memory order.  The final per-group sums [4][1024]
// reuse the buffers.
template <typename T>
__host__ __device__ constexpr int rd_tile() {
    return 64 * (RD_P + ad_pad<T>());
}
template <typename T>
__host__ __device__ inline size_t reduce_dense_smem(int nchunked) {
    return (size_t)RD_S * (rd_tile<T>() + nchunked * 32 * RD_P) * sizeof(T);
}

// Operand modes (X in bits 0-1, Z in bits 2-3): 0 one entry per copy,
// 1 four consecutive positions per copy, 3 the tile's 16-byte chunks in
// memory order (planned table), scattered into the tile's rows.
template <typename T>
__global__ void __launch_bounds__(256) k_reduce_dense(const __grid_constant__ RDesc d, int modes,
                                                      int64_t chunk, int nchunks, T *part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int RR = RD_P + ad_pad<T>();
    const int mx_ = modes & 3, mz_ = (modes >> 2) & 3;
    const int nchunked = (mx_ == 3) + (mz_ == 3);
    const int TB = rd_tile<T>() + nchunked * 32 * RD_P;   // one buffer
    T *Ts = (T *)smraw;
    const int tid = threadIdx.x;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *tz = d.tab + nin;
    const int nod = d.nmd - d.nin_d;
    const int64_t g = (int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (g >= d.ng * d.nbeta) return;
    const int64_t beta = g / d.ng, gi = g - beta * d.ng;
    int64_t gx = beta * d.bsx, gz = beta * d.bsz, go = 0;
    group_offsets(d, gi, gx, gz, go);
    const T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    const T sz = d.mxz ? pow2neg<T>(exp_of_bits(d.mxz[beta * d.mxz_bs])) : T(1);
    const int64_t cper = (nin + RD_P - 1) / RD_P;
    const int64_t ntile = d.nouter * cper;
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = t0 + chunk < ntile ? t0 + chunk : ntile;
    const int nk = t1 > t0 ? (int)(t1 - t0) : 0;
    const int lcper = log2_if_pow2(cper);
    const T *X = (const T *)d.X, *Z = (const T *)d.Z;
    const uint32_t ts0 = (uint32_t)__cvta_generic_to_shared(Ts);
    // staging of operand h (chunk mode) inside a buffer, after the tile
    auto stage_off = [&](int h) { return rd_tile<T>() + (h == 1 && mx_ == 3 ? 32 * RD_P : 0); };
    // chunk modes: this thread's chunks q = tid + 256 r (r < 2) of each operand,
    // the same in every tile, kept in registers
    int32_t crel[2][2];
    uint2 csl[2][2];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int nq = (h ? d.nt : d.ns) * (RD_P / 4), q = tid + 256 * r;
            const int32_t at = h ? d.czo : d.cxo;
            crel[h][r] = 0;
            csl[h][r] = make_uint2(0u, 0u);
            if ((h ? mz_ : mx_) == 3 && q < nq) {
                crel[h][r] = __ldg(d.tab + at + q);
                csl[h][r] = __ldg((const uint2 *)(d.tab + at + nq) + q);
            }
        }
    auto issue = [&](int k, int b) {
        if (k < nk) {
            int64_t crem;
            const int64_t o = div_tile(t0 + k, cper, lcper, crem);
            int64_t cbx = gx, cbz = gz;
            reduce_outer(d, o, nod, cbx, cbz);
            const int j0 = (int)crem * RD_P;
            const uint32_t sb = ts0 + (uint32_t)(b * TB * sizeof(T));
            // X rows 0..31, Z rows 32..63
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const T *base = h ? Z + cbz : X + cbx;
                const int *tab = h ? tz : tx;
                const int nv = h ? d.nt : d.ns;
                const int md = h ? mz_ : mx_;
                if (md == 3) {
                    const T *bt = base + __ldg(tab + j0);
                    const uint32_t st = sb + (uint32_t)(stage_off(h) * sizeof(T));
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const int q = tid + 256 * r;
                        if (q < nv * (RD_P / 4))
                            cp_async4<T>(st + (uint32_t)(4 * q * sizeof(T)), bt + crel[h][r], true);
                    }
                } else if (md == 1) {
                    for (int e = tid; e < 32 * (RD_P / 4); e += 256) {
                        const int v = e / (RD_P / 4), p = (e % (RD_P / 4)) * 4;
                        const int j = j0 + p;
                        const bool ok = v < nv && j < nin;
                        const int64_t off = h ? d.zoff[v] : d.xoff[v];
                        cp_async4<T>(sb + (uint32_t)(((32 * h + v) * RR + p) * sizeof(T)),
                                     ok ? base + __ldg(tab + j) + off : base, ok);
                    }
                } else {
                    for (int e = tid; e < 32 * RD_P; e += 256) {
                        const int v = e / RD_P, p = e % RD_P;
                        const int j = j0 + p;
                        const bool ok = v < nv && j < nin;
                        const int64_t off = h ? d.zoff[v] : d.xoff[v];
                        cp_async1<T>(sb + (uint32_t)(((32 * h + v) * RR + p) * sizeof(T)),
                                     ok ? base + __ldg(tab + j) + off : base, ok);
                    }
                }
            }
        }
        cp_async_commit();
    };
    // thread: positions [16 pq, 16 pq + 16) of each tile, outputs
    // s = ts + 8 i, t = tt + 8 j (i, j < 4)
    const int pq = tid >> 6, ts = (tid >> 3) & 7, tt = tid & 7;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    issue(0, 0);
    issue(1, 1);
    int b = 0;
    for (int k = 0; k < nk; ++k) {
        cp_async_wait<1>();
        __syncthreads();
        issue(k + 2, b == 0 ? 2 : b - 1);
        T *tb = Ts + b * TB;
        if (nchunked) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if ((h ? mz_ : mx_) != 3) continue;
                const int nq = (h ? d.nt : d.ns) * (RD_P / 4);
                const T *st = tb + stage_off(h);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = tid + 256 * r;
                    if (q < nq) {
                        T v[4];
                        ld4(st + 4 * q, v);
                        scatter4(tb, csl[h][r], v);
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = 16 * pq + 4 * q;
            T xv[4][4], zv[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ld4(tb + (ts + 8 * i) * RR + p, xv[i]);
#pragma unroll
            for (int j = 0; j < 4; ++j) ld4(tb + (32 + tt + 8 * j) * RR + p, zv[j]);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += xv[i][u] * zv[j][u];
        }
        b = b == 2 ? 0 : b + 1;
    }
    cp_async_wait<0>();
    __syncthreads();
    // the four position groups' sums, then this block's partial row
    T *red = Ts;   // [4][1024]
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[pq * 1024 + (ts + 8 * i) * 32 + tt + 8 * j] = acc[i][j];
    __syncthreads();
    const T scale = sx * sz;
    T *prow = part + (g * nchunks + blockIdx.x) * 1024;
    for (int o = tid; o < 1024; o += 256)
        prow[o] = ((red[o] + red[1024 + o]) + (red[2048 + o] + red[3072 + o])) * scale;
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (tid == 0) last = atomicAdd(d.cnt + g, 1u) == (unsigned)(nchunks - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const T *pg = part + g * nchunks * 1024;
    T mx = 0;
    for (int o = tid; o < 1024; o += 256) {
        const int s = o >> 5, t = o & 31;
        T v = 0;
        for (int c = 0; c < nchunks; ++c) v += __ldcg(pg + (int64_t)c * 1024 + o);
        if (s < d.ns && t < d.nt) {
            ((T *)d.O)[go + beta * d.bso + d.oso[s] + d.oto[t]] = v;
            mx = mx > v ? mx : v;
        }
    }
    if (d.mxo) block_max_atomic(d.mxo + beta, (double)mx);
    if (tid == 0) d.cnt[g] = 0u;
}

}  // namespace tn

// Streaming kernels for the HBM-bound pairwise contractions of a contraction
// tree (the "big tensor x small tensor" absorptions and the reductions of two
// big tensors to a small one, which dominate a tree's read-write complexity,
// paper Sec. Benchmarks).  Each big operand is read from HBM exactly once:
//
//   k_absorb       one thread per position r kept from the streamed operand X;
//                  it loads X[r, s] for every summed combination s into
//                  registers and writes Y[t, r] for every new combination t
//                  from the small operand W (read through L1).  Sum-product
//                  with power-of-two rescaling, or max-plus with the flat index
//                  of the maximiser (Eq. tropical).
//   k_reduce_part  each block streams a chunk of the summed positions m of one
//                  group g and accumulates the outer products X[g,m,s] Z[g,m,t]
//                  in registers; the group's last block to finish sums the
//                  chunk partials in a fixed order (deterministic), writes the
//                  result and records its maximum.
//   k_reduce_vec   the same reduction where the fastest summed dim is
//                  contiguous in both operands: 16-byte vector loads straight
//                  into registers instead of per-element staged copies.
#include <cmath>

#pragma once
#include <algorithm>
#include <mutex>
#include <vector>

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
    if (SEMI == SUM) {
        T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
        T sw = d.mxw ? pow2neg<T>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : T(1);
        scale = sx * sw;
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
                    x[u][s] = (on[u] && (NS == 1 || s < d.ns)) ? Xb[ox + d.xoff[s]] : T(0);
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
                            T v = x[u][s] + __ldg(W + d.wso[s] + d.wto[t]);
                            if (v > best) { best = v; bk = s; }
                        }
                        Y[d.yoff[t]] = best;
                        if (d.argmax) d.argmax[by + oy[u] + d.yoff[t]] = bk;
                    }
                }
            }
        }
    }
    if (SEMI == SUM && d.mxy) block_max_atomic(d.mxy + beta, (double)mx * (double)scale);
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

template <typename T, int NS, int NT>
static void absorb_go(const ADesc &d, int semiring, cudaStream_t st) {
    constexpr int BLK = absorb_blk<T, NS, NT>();
    const size_t smem = (size_t)d.nsh * BLK * sizeof(T);
    if constexpr (NS * NT >= 16) {
        if (semiring == SUM && smem <= 32768) {
            // a few resident blocks per SM, each stages W once
            constexpr int U = NS * NT <= 64 ? 2 : 1;
            int64_t ntile = d.nouter * ((d.nin + 256 * U - 1) / (256 * U));
            int64_t cap = std::max<int64_t>(1, (152LL * 4) / std::max(1, d.nbeta));
            dim3 grid((unsigned)std::max<int64_t>(1, std::min(ntile, cap)), (unsigned)d.nbeta, 1);
            k_absorb_sm<T, NS, NT><<<grid, 256, smem, st>>>(d);
            return;
        }
    }
    constexpr int U = NS * NT <= 4 ? 8 : NS * NT <= 16 ? 4 : NS * NT <= 64 ? 2 : 1;
    int64_t ntile = d.nouter * ((d.nin + 256 * U - 1) / (256 * U));
    int64_t cap = std::max<int64_t>(1, (152LL * 16) / std::max(1, d.nbeta));
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

template <typename T>
void launch_absorb(const ADesc &d0, int semiring, cudaStream_t st) {
    if (d0.nr * d0.nbeta == 0) return;
    ADesc d = d0;
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

// ------------------------------------------------------------------ reduce

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

// Block epilogue of the reduce kernels: per-warp sums of the accumulators (a
// warp lies inside one sub-block), then per sub-block, written as this
// block's partial; the group's last block to finish sums the partials of all
// nchunks blocks in a fixed order (deterministic), writes O, records its
// maximum and re-arms the group's counter.
template <typename T, int NS, int NT>
__device__ __forceinline__ void reduce_finish(const RDesc &d, T (&acc)[NS][NT], int64_t g,
                                              int64_t beta, int64_t gi, int nbs, int nbt,
                                              int nchunks, int pstride, T scale, T *part) {
    __shared__ T red[8][NS * NT];
    __shared__ bool last;
    const int nb = nbs * nbt, pp = 256 / nb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            T v = acc[s][t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[w][s * NT + t] = v;
        }
    __syncthreads();
    const int wper = pp / 32;
    for (int i = threadIdx.x; i < nb * NS * NT; i += blockDim.x) {
        const int b = i / (NS * NT), ii = i - b * (NS * NT);
        T v = 0;
        for (int q = 0; q < wper; ++q) v += red[b * wper + q][ii];
        part[(g * nchunks + blockIdx.x) * pstride + i] = v * scale;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(d.cnt + g, 1u) == (unsigned)(nchunks - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    T mx = 0;
    int64_t ox = 0, oz = 0, oo = beta * d.bso;
    group_offsets(d, gi, ox, oz, oo);
    for (int i = w; i < nb * NS * NT; i += (int)(blockDim.x >> 5)) {
        const int b = i / (NS * NT), ii = i - b * (NS * NT);
        const int s = (b / nbt) * NS + ii / NT, t = (b % nbt) * NT + ii % NT;
        if (s >= d.ns || t >= d.nt) continue;
        T v = 0;
        for (int c = lane; c < nchunks; c += 32) v += __ldcg(part + (g * nchunks + c) * pstride + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            ((T *)d.O)[oo + d.oso[s] + d.oto[t]] = v;
            mx = mx > v ? mx : v;
        }
    }
    if (d.mxo) block_max_atomic(d.mxo + beta, (double)mx);
    if (threadIdx.x == 0) d.cnt[g] = 0u;
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

// The summed positions m split into inner ones (offset table computed at plan
// time, at most A_INNER) and outer ones.  A block's 256 threads form nb =
// nbs x nbt sub-blocks of pp = 256 / nb threads: thread (b, p) owns position p
// of every staged tile and the NS x NT outputs (bs NS + s, bt NT + t) of its
// sub-block b = (bs, bt), so outputs up to 32 x 32 need one pass over the
// operands (threads of different sub-blocks fetch the same position's values
// separately; the repeats hit L1).  Each thread's operand values for tiles of
// pp positions (outer index, inner chunk) come into its own shared-memory
// slots by asynchronous copies red_stages() tiles ahead of use (no barrier);
// blocks take contiguous tile ranges of one group, write per-block partials,
// and the group's last block to finish sums them in a fixed order
// (deterministic), writes O and records its maximum.
template <typename T>
__host__ __device__ constexpr int red_stages() {
    return sizeof(T) == 8 ? 3 : 4;
}


template <typename T, int NS, int NT>
__global__ void __launch_bounds__(256) k_reduce_part(const __grid_constant__ RDesc d, int nbs,
                                                     int nbt, int64_t chunk, int nchunks,
                                                     int pstride, T *part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int S = red_stages<T>(), W = NS + NT;
    // [S][W][256]: each thread stages (and later reads) only its own slots
    T *buf = (T *)smraw + threadIdx.x;
    const int nb = nbs * nbt, pp = 256 / nb;
    const int sub = threadIdx.x / pp, p = threadIdx.x - sub * pp;
    const int bs = sub / nbt, bt = sub - bs * nbt;
    const int nin = (int)d.nin;
    const int *tx = d.tab, *tz = d.tab + nin;
    const int nod = d.nmd - d.nin_d;
    int64_t g = (int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (g >= d.ng * d.nbeta) return;
    int64_t beta = g / d.ng, gi = g - beta * d.ng;
    int64_t gx = beta * d.bsx, gz = beta * d.bsz, go = 0;
    group_offsets(d, gi, gx, gz, go);
    T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    T sz = d.mxz ? pow2neg<T>(exp_of_bits(d.mxz[beta * d.mxz_bs])) : T(1);
    T acc[NS][NT];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[s][t] = 0;
    const int64_t cper = (nin + pp - 1) / pp;
    const int64_t ntile = d.nouter * cper;
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = t0 + chunk < ntile ? t0 + chunk : ntile;
    const int nk = t1 > t0 ? (int)(t1 - t0) : 0;
    const T *X = (const T *)d.X, *Z = (const T *)d.Z;
    const int s0 = bs * NS, z0 = bt * NT;
    const int lcper = log2_if_pow2(cper);
    int64_t cur_o = -1, cbx = 0, cbz = 0;   // outer decode of the last tile
    auto issue = [&](int k) {
        T *sb = buf + (k % S) * W * 256;
        const int64_t tile = t0 + k;
        int64_t crem;
        const int64_t o = div_tile(tile, cper, lcper, crem);
        const int j = (int)crem * pp + p;
        if (o != cur_o) {
            cur_o = o;
            cbx = gx;
            cbz = gz;
            reduce_outer(d, o, nod, cbx, cbz);
        }
        if (j < nin) {
            const T *xp = X + cbx + __ldg(tx + j);
            const T *zp = Z + cbz + __ldg(tz + j);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (s0 + s < d.ns) cp_async_el(sb + s * 256, xp + d.xoff[s0 + s]);
                else sb[s * 256] = T(0);
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (z0 + t < d.nt) cp_async_el(sb + (NS + t) * 256, zp + d.zoff[z0 + t]);
                else sb[(NS + t) * 256] = T(0);
            }
        } else {
#pragma unroll
            for (int w = 0; w < W; ++w) sb[w * 256] = T(0);
        }
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        if (k < nk) issue(k);
        cp_async_commit();
    }
    for (int k = 0; k < nk; ++k) {
        if (k + S - 1 < nk) issue(k + S - 1);
        cp_async_commit();
        cp_async_wait<S - 1>();
        const T *sb = buf + (k % S) * W * 256;
        T x[NS], z[NT];
#pragma unroll
        for (int s = 0; s < NS; ++s) x[s] = sb[s * 256];
#pragma unroll
        for (int t = 0; t < NT; ++t) z[t] = sb[(NS + t) * 256];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int t = 0; t < NT; ++t) acc[s][t] += x[s] * z[t];
    }
    cp_async_wait<0>();
    reduce_finish<T, NS, NT>(d, acc, g, beta, gi, nbs, nbt, nchunks, pstride, sx * sz, part);
}

// Vector form of the reduce for nodes whose fastest summed dim has stride 1
// in both operands and every other offset is a multiple of VW = 16 /
// sizeof(T) elements (reduce_vec_shape, plus 16-byte aligned operands): a
// tile is U x pp groups of VW consecutive positions (outer index, inner
// chunk); thread (b, p) loads, for each of its U groups, the NS values of X
// and NT values of Z as 16-byte vectors straight into registers and
// accumulates their VW outer products.  A position then costs (NS + NT) / VW
// loads and no staging, against NS + NT copies and shared-memory reads in
// k_reduce_part; same sub-blocks, partials and finalize.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ void fma_vec(float &a, const float4 &x, const float4 &z) {
    a = fmaf(x.x, z.x, a);
    a = fmaf(x.y, z.y, a);
    a = fmaf(x.z, z.z, a);
    a = fmaf(x.w, z.w, a);
}
__device__ __forceinline__ void fma_vec(double &a, const double2 &x, const double2 &z) {
    a = fma(x.x, z.x, a);
    a = fma(x.y, z.y, a);
}
__device__ __forceinline__ void vzero(float4 &v) { v = make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ void vzero(double2 &v) { v = make_double2(0.0, 0.0); }

// Groups of VW positions a thread loads per tile, by its number of outputs.
__host__ __device__ constexpr int red_vec_groups(int nout) {
    return nout >= 32 ? 1 : 2;
}

template <typename T, int NS, int NT>
__global__ void __launch_bounds__(256, NS * NT >= 64 ? 1 : 2) k_reduce_vec(const __grid_constant__ RDesc d, int nbs,
                                                    int nbt, int64_t chunk, int nchunks,
                                                    int pstride, T *part) {
    using V = typename Vec16<T>::type;
    constexpr int VW = 16 / (int)sizeof(T), U = red_vec_groups(NS * NT);
    const int nb = nbs * nbt, pp = 256 / nb;
    const int sub = threadIdx.x / pp, p = threadIdx.x - sub * pp;
    const int bs = sub / nbt, bt = sub - bs * nbt;
    const int nin = (int)d.nin, nq = nin / VW;
    const int *tx = d.tab, *tz = d.tab + nin;
    const int nod = d.nmd - d.nin_d;
    int64_t g = (int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (g >= d.ng * d.nbeta) return;
    int64_t beta = g / d.ng, gi = g - beta * d.ng;
    int64_t gx = beta * d.bsx, gz = beta * d.bsz, go = 0;
    group_offsets(d, gi, gx, gz, go);
    T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    T sz = d.mxz ? pow2neg<T>(exp_of_bits(d.mxz[beta * d.mxz_bs])) : T(1);
    T acc[NS][NT];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[s][t] = 0;
    const int64_t cper = (nq + pp * U - 1) / (pp * U);
    const int64_t ntile = d.nouter * cper;
    const int64_t t0 = (int64_t)blockIdx.x * chunk;
    const int64_t t1 = t0 + chunk < ntile ? t0 + chunk : ntile;
    const T *X = (const T *)d.X, *Z = (const T *)d.Z;
    const int s0 = bs * NS, z0 = bt * NT;
    const int lcper = log2_if_pow2(cper);
    int64_t cur_o = -1, cbx = 0, cbz = 0;   // outer decode of the last tile
    for (int64_t tile = t0; tile < t1; ++tile) {
        int64_t crem;
        const int64_t o = div_tile(tile, cper, lcper, crem);
        if (o != cur_o) {
            cur_o = o;
            cbx = gx;
            cbz = gz;
            reduce_outer(d, o, nod, cbx, cbz);
        }
        V xv[U][NS], zv[U][NT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = ((int)crem * U + u) * pp + p;
            const bool ok = q < nq;
            const int j = ok ? q * VW : 0;
            const T *xp = X + cbx + __ldg(tx + j);
            const T *zp = Z + cbz + __ldg(tz + j);
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                if (ok && s0 + s < d.ns) xv[u][s] = __ldg((const V *)(xp + d.xoff[s0 + s]));
                else vzero(xv[u][s]);
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                if (ok && z0 + t < d.nt) zv[u][t] = __ldg((const V *)(zp + d.zoff[z0 + t]));
                else vzero(zv[u][t]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int t = 0; t < NT; ++t) fma_vec(acc[s][t], xv[u][s], zv[u][t]);
    }
    reduce_finish<T, NS, NT>(d, acc, g, beta, gi, nbs, nbt, nchunks, pstride, sx * sz, part);
}

static int pow2ceil_i(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Can the node take k_reduce_vec with VW-element vectors (pointers aside)?
// The fastest summed dim must have stride 1 in X and Z and a size divisible by
// VW, and every other offset of X and Z a multiple of VW, so that the VW
// positions of a group are consecutive in both operands and each vector
// starts on a VW-element boundary of the operand.
static bool reduce_vec_shape(const RDesc &d, int vw) {
    if (d.nin_d < 1 || d.nmd < 1) return false;
    const int k = d.nmd - 1;
    if (d.msx[k] != 1 || d.msz2[k] != 1 || d.msz[k] % vw) return false;
    auto mult = [vw](int64_t v) { return v % vw == 0; };
    for (int i = 0; i < k; ++i)
        if (!mult(d.msx[i]) || !mult(d.msz2[i])) return false;
    for (int i = 0; i < d.ngd; ++i)
        if (!mult(d.gsx[i]) || !mult(d.gsz2[i])) return false;
    for (int i = 0; i < d.ns; ++i)
        if (!mult(d.xoff[i])) return false;
    for (int i = 0; i < d.nt; ++i)
        if (!mult(d.zoff[i])) return false;
    return mult(d.bsx) && mult(d.bsz);
}

// One launch's shape: per-thread sub-block NS x NT (<= 8 x 8), nbs x nbt
// sub-blocks (<= 8), the s range it covers, the chunking of the tiles for
// k_reduce_part and, where the node's shape allows it (vec), for
// k_reduce_vec.
struct RedPiece {
    int NS, NT, nbs, nbt, s0, ns;
    int64_t chunk;
    int nchunks, pstride;
    bool vec;
    int64_t vchunk;
    int vnchunks;
};

static std::vector<RedPiece> reduce_pieces(const RDesc &d, int esz) {
    std::vector<RedPiece> out;
    RedPiece p{};
    p.NS = d.ns <= 1 ? 1 : d.ns <= 2 ? 2 : d.ns <= 4 ? 4 : 8;
    p.NT = d.nt <= 1 ? 1 : d.nt <= 2 ? 2 : d.nt <= 4 ? 4 : 8;
    p.nbt = pow2ceil_i((d.nt + p.NT - 1) / p.NT);
    int nbs_all = pow2ceil_i((d.ns + p.NS - 1) / p.NS);
    p.nbs = std::min(nbs_all, 8 / p.nbt);
    const int pp = 256 / (p.nbs * p.nbt);
    const int64_t groups = d.ng * d.nbeta;
    const int64_t ntile = d.nouter * ((d.nin + pp - 1) / pp);
    // about two resident blocks per SM in total
    const int64_t want = std::max<int64_t>(1, (152LL * 2) / std::max<int64_t>(1, groups));
    p.chunk = std::max<int64_t>(1, (ntile + want - 1) / want);
    p.nchunks = (int)((ntile + p.chunk - 1) / p.chunk);
    p.pstride = p.nbs * p.nbt * p.NS * p.NT;
    // FP64 keeps the vector form to <= 32 outputs a thread (registers)
    const int vw = 16 / esz;
    p.vec = reduce_vec_shape(d, vw) && (esz == 4 || p.NS * p.NT <= 32);
    if (p.vec) {
        const int64_t per = (int64_t)pp * red_vec_groups(p.NS * p.NT);
        const int64_t vtile = d.nouter * ((d.nin / vw + per - 1) / per);
        p.vchunk = std::max<int64_t>(1, (vtile + want - 1) / want);
        p.vnchunks = (int)((vtile + p.vchunk - 1) / p.vchunk);
    }
    for (int s0 = 0; s0 < d.ns; s0 += p.nbs * p.NS) {
        p.s0 = s0;
        p.ns = std::min(p.nbs * p.NS, d.ns - s0);
        out.push_back(p);
    }
    return out;
}

#ifdef TN_STREAM_HOST_DEFS
size_t reduce_scratch_bytes(const RDesc &d, int elem_bytes) {
    size_t mx = 0;
    for (auto &p : reduce_pieces(d, elem_bytes)) {
        const int nch = std::max(p.nchunks, p.vec ? p.vnchunks : 0);
        mx = std::max(mx, (size_t)(d.ng * d.nbeta * nch) * p.pstride * elem_bytes);
    }
    return mx;
}
#endif

template <typename T, int NS, int NT>
static void reduce_go(const RDesc &d, const RedPiece &p, void *scratch, cudaStream_t st) {
    const int64_t groups = d.ng * d.nbeta;
    // the vector form also needs both operands on 16-byte boundaries
    constexpr bool kvec = sizeof(T) == 4 || NS * NT <= 32;
    const bool vec = kvec && p.vec && ((uintptr_t)d.X % 16) == 0 && ((uintptr_t)d.Z % 16) == 0;
    const int nch = vec ? p.vnchunks : p.nchunks;
    dim3 grid((unsigned)nch, (unsigned)std::min<int64_t>(groups, 65535),
              (unsigned)((groups + 65534) / 65535));
    if constexpr (kvec) {
        if (vec) {
            k_reduce_vec<T, NS, NT><<<grid, 256, 0, st>>>(d, p.nbs, p.nbt, p.vchunk, nch,
                                                          p.pstride, (T *)scratch);
            return;
        }
    }
    constexpr size_t smem = (size_t)red_stages<T>() * (NS + NT) * 256 * sizeof(T);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_reduce_part<T, NS, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    });
    k_reduce_part<T, NS, NT><<<grid, 256, smem, st>>>(d, p.nbs, p.nbt, p.chunk, nch, p.pstride,
                                                      (T *)scratch);
}

template <typename T, int NS>
static void reduce_nt(const RDesc &d, const RedPiece &p, void *scratch, cudaStream_t st) {
    if (p.NT == 1) reduce_go<T, NS, 1>(d, p, scratch, st);
    else if (p.NT == 2) reduce_go<T, NS, 2>(d, p, scratch, st);
    else if (p.NT == 4) reduce_go<T, NS, 4>(d, p, scratch, st);
    else reduce_go<T, NS, 8>(d, p, scratch, st);
}

// Outputs with more than 8 sub-blocks run as several launches over ranges of
// s (each reads its slice of X and all of Z).
template <typename T>
void launch_reduce(const RDesc &d, void *scratch, cudaStream_t st) {
    if (d.ng * d.nbeta == 0) return;
    for (const RedPiece &p : reduce_pieces(d, (int)sizeof(T))) {
        RDesc c = d;
        c.ns = p.ns;
        for (int i = 0; i < c.ns; ++i) {
            c.xoff[i] = d.xoff[p.s0 + i];
            c.oso[i] = d.oso[p.s0 + i];
        }
        if (p.NS == 1) reduce_nt<T, 1>(c, p, scratch, st);
        else if (p.NS == 2) reduce_nt<T, 2>(c, p, scratch, st);
        else if (p.NS == 4) reduce_nt<T, 4>(c, p, scratch, st);
        else reduce_nt<T, 8>(c, p, scratch, st);
    }
}

#ifdef TN_STREAM_HOST_DEFS
int reduce_launches(const RDesc &d) { return (int)reduce_pieces(d, 4).size(); }
bool reduce_vector_form(const RDesc &d, int elem_bytes) {
    const auto pieces = reduce_pieces(d, elem_bytes);
    return !pieces.empty() && pieces[0].vec && ((uintptr_t)d.X % 16) == 0 &&
           ((uintptr_t)d.Z % 16) == 0;
}
#endif


}  // namespace tn

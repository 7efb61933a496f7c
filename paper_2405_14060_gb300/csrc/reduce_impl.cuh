// Streaming reductions of two big tensors to a small one (the B-bar =
// con(A, C-bar) steps of the adjoint sweep, Thm. "Tensor network
// differentiation", Eq. einback, and forward nodes whose result is small).
// Both big operands are read from HBM exactly once:
//
//   k_reduce_part  each block streams a chunk of the summed positions m of one
//                  group g and accumulates the outer products X[g,m,s] Z[g,m,t]
//                  in registers; the group's last block to finish sums the
//                  chunk partials in a fixed order (deterministic), writes the
//                  result and records its maximum.
//   k_reduce_vec   the same reduction where the fastest summed dim is
//                  contiguous in both operands: 16-byte vector loads straight
//                  into registers instead of per-element staged copies.
#pragma once
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "dense_impl.cuh"
#include "devutil.cuh"
#include "stream.cuh"

namespace tn {

// 16-byte vectors of T and the few operations the reduce kernels need on them.
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
__device__ __forceinline__ void vadd(float4 &a, const float4 &b) {
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
}
__device__ __forceinline__ void vadd(double2 &a, const double2 &b) {
    a.x += b.x;
    a.y += b.y;
}

// Block epilogue of the reduce kernels: per-warp sums of the accumulators (a
// warp lies inside one sub-block), then per sub-block, written as this
// block's row of pstride partials; the group's last block to finish sums the
// nchunks rows, writes O, records its maximum and re-arms the group's
// counter.  In that sum thread t takes the column group t % ncol (CW
// consecutive partials, one 16-byte load per row when pstride allows) over
// the rows q, q + nsplit, ... (q = t / ncol), so all 256 threads load whole
// rows at once; the nsplit sums of a column are then added in order of q.
// The order is fixed by the launch shape, so the result is deterministic.
template <typename T, int NS, int NT>
__device__ __forceinline__ void reduce_finish(const RDesc &d, T (&acc)[NS][NT], int64_t g,
                                              int64_t beta, int64_t gi, int nbs, int nbt,
                                              int nchunks, int pstride, T scale, T *part) {
    using V = typename Vec16<T>::type;
    constexpr int CW = 16 / (int)sizeof(T);
    __shared__ T red[8][NS * NT];
    __shared__ __align__(16) T fin[256 * CW];
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
    // pstride is a power of two <= 512: ncol divides 256 or is a multiple of it
    const T *pg = part + g * nchunks * pstride;
    const bool vec = pstride % CW == 0 && ((uintptr_t)pg % 16) == 0;
    const int ncol = vec ? pstride / CW : pstride;
    const int nsplit = ncol >= 256 ? 1 : 256 / ncol;
    const int q = threadIdx.x / ncol;
    for (int col = threadIdx.x % ncol; col < ncol; col += 256) {
        if (vec) {
            V a0, a1;
            vzero(a0);
            vzero(a1);
            int c = q;
#pragma unroll 4
            for (; c + nsplit < nchunks; c += 2 * nsplit) {
                const V v0 = __ldcg((const V *)(pg + (int64_t)c * pstride) + col);
                const V v1 = __ldcg((const V *)(pg + (int64_t)(c + nsplit) * pstride) + col);
                vadd(a0, v0);
                vadd(a1, v1);
            }
            if (c < nchunks) vadd(a0, __ldcg((const V *)(pg + (int64_t)c * pstride) + col));
            vadd(a0, a1);
            *(V *)(fin + q * pstride + col * CW) = a0;
        } else {
            T a0 = 0, a1 = 0;
            int c = q;
#pragma unroll 4
            for (; c + nsplit < nchunks; c += 2 * nsplit) {
                a0 += __ldcg(pg + (int64_t)c * pstride + col);
                a1 += __ldcg(pg + (int64_t)(c + nsplit) * pstride + col);
            }
            if (c < nchunks) a0 += __ldcg(pg + (int64_t)c * pstride + col);
            fin[q * pstride + col] = a0 + a1;
        }
    }
    __syncthreads();
    T mx = 0;
    int64_t ox = 0, oz = 0, oo = beta * d.bso;
    group_offsets(d, gi, ox, oz, oo);
    for (int i = threadIdx.x; i < pstride; i += blockDim.x) {
        T v = 0;
        for (int k = 0; k < nsplit; ++k) v += fin[k * pstride + i];
        const int b = i / (NS * NT), ii = i - b * (NS * NT);
        const int s = (b / nbt) * NS + ii / NT, t = (b % nbt) * NT + ii % NT;
        if (s < d.ns && t < d.nt) {
            ((T *)d.O)[oo + d.oso[s] + d.oto[t]] = v;
            mx = mx > v ? mx : v;
        }
    }
    if (d.mxo) block_max_atomic(d.mxo + beta, (double)mx);
    if (threadIdx.x == 0) d.cnt[g] = 0u;
}

// The summed positions m split into inner ones (offset table computed at plan
// time, at most 2048) and outer ones.  A block's 256 threads form nb =
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
        // as many blocks as fit at once: one per SM with 64 FP32 outputs a
        // thread (its registers), else two
        const int64_t vwant = std::max<int64_t>(
            1, (152LL * (p.NS * p.NT >= 64 ? 1 : 2)) / std::max<int64_t>(1, groups));
        const int64_t per = (int64_t)pp * red_vec_groups(p.NS * p.NT);
        const int64_t vtile = d.nouter * ((d.nin / vw + per - 1) / per);
        p.vchunk = std::max<int64_t>(1, (vtile + vwant - 1) / vwant);
        p.vnchunks = (int)((vtile + p.vchunk - 1) / p.vchunk);
    }
    for (int s0 = 0; s0 < d.ns; s0 += p.nbs * p.NS) {
        p.s0 = s0;
        p.ns = std::min(p.nbs * p.NS, d.ns - s0);
        out.push_back(p);
    }
    return out;
}

// Dense form (k_reduce_dense): more than 256 outputs per group after
// rounding to powers of two.  Its chunking: about three resident blocks per
// SM over all groups.
static bool reduce_dense_form(const RDesc &d) {
    return pow2ceil_i(d.ns) * pow2ceil_i(d.nt) > 256;
}
static void reduce_dense_shape(const RDesc &d, int64_t &chunk, int &nchunks) {
    const int64_t groups = std::max<int64_t>(1, d.ng * d.nbeta);
    const int64_t ntile = d.nouter * ((d.nin + RD_P - 1) / RD_P);
    const int64_t want = std::max<int64_t>(1, (152LL * 3) / groups);
    chunk = std::max<int64_t>(1, (ntile + want - 1) / want);
    nchunks = (int)std::max<int64_t>(1, (ntile + chunk - 1) / chunk);
}
// 16-byte copies of four consecutive positions (bit 0: X, bit 1: Z) where
// every aligned quad of positions is contiguous and 16-byte aligned.
static int reduce_dense_vm(const RDesc &d) {
    const int L = d.nmd - 1;   // the fastest summed dim
    auto ok = [&](const void *p, int64_t bs, const int64_t *ms, const int64_t *gs,
                  const int64_t *off, int n) {
        if (((uintptr_t)p & 15) || bs % 4 || d.nin % 4 || d.msz[L] % 4 || ms[L] != 1) return false;
        for (int k = 0; k < L; ++k)
            if (ms[k] % 4) return false;
        for (int k = 0; k < d.ngd; ++k)
            if (gs[k] % 4) return false;
        for (int i = 0; i < n; ++i)
            if (off[i] % 4) return false;
        return true;
    };
    return (ok(d.X, d.bsx, d.msx, d.gsx, d.xoff, d.ns) ? 1 : 0) |
           (ok(d.Z, d.bsz, d.msz2, d.gsz2, d.zoff, d.nt) ? 2 : 0);
}

// Operand modes of k_reduce_dense: four positions per copy where possible,
// else the planned chunk table, else one entry per copy.
static int reduce_dense_modes(const RDesc &d) {
    const int vm = reduce_dense_vm(d);
    const int mx = (vm & 1) ? 1 : d.cx ? 3 : 0;
    const int mz = (vm & 2) ? 1 : d.cz ? 3 : 0;
    return mx | (mz << 2);
}

template <typename T>
static void reduce_dense_go(const RDesc &d, void *scratch, cudaStream_t st) {
    const int64_t groups = d.ng * d.nbeta;
    int64_t chunk;
    int nchunks;
    reduce_dense_shape(d, chunk, nchunks);
    const int modes = reduce_dense_modes(d);
    const size_t smem = reduce_dense_smem<T>(((modes & 3) == 3) + (((modes >> 2) & 3) == 3));
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_reduce_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)reduce_dense_smem<T>(2));
    });
    dim3 grid((unsigned)nchunks, (unsigned)std::min<int64_t>(groups, 65535),
              (unsigned)((groups + 65534) / 65535));
    k_reduce_dense<T><<<grid, 256, smem, st>>>(d, modes, chunk, nchunks, (T *)scratch);
}

#ifdef TN_STREAM_HOST_DEFS
size_t reduce_scratch_bytes(const RDesc &d, int elem_bytes) {
    if (reduce_dense_form(d)) {
        int64_t chunk;
        int nchunks;
        reduce_dense_shape(d, chunk, nchunks);
        return (size_t)(d.ng * d.nbeta * nchunks) * 1024 * (size_t)elem_bytes;
    }
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
    if (reduce_dense_form(d)) {
        reduce_dense_go<T>(d, scratch, st);
        return;
    }
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
int reduce_dense_describe(const RDesc &d) { return reduce_dense_form(d) ? reduce_dense_modes(d) : -1; }
int reduce_launches(const RDesc &d) {
    return reduce_dense_form(d) ? 1 : (int)reduce_pieces(d, 4).size();
}
bool reduce_vector_form(const RDesc &d, int elem_bytes) {
    if (reduce_dense_form(d)) return reduce_dense_vm(d) == 3;
    const auto pieces = reduce_pieces(d, elem_bytes);
    return !pieces.empty() && pieces[0].vec && ((uintptr_t)d.X % 16) == 0 &&
           ((uintptr_t)d.Z % 16) == 0;
}
#endif

}  // namespace tn

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
//                  in registers; k_reduce_fin sums the chunk partials in a
//                  fixed order (deterministic) and records the maxima.
#include <cmath>

#pragma once
#include <algorithm>

#include "devutil.cuh"
#include "stream.cuh"

namespace tn {

// Positions are processed in tiles of TILE consecutive inner positions of one
// outer position: the outer offsets are decoded once per tile (64-bit), the
// inner ones per position in 32-bit arithmetic, and every thread issues the
// loads of TILE / blockDim positions before using them.
constexpr int A_TILE = 1024;

// NS / NT are the exact numbers of summed / new combinations.  Sum-product
// accumulates the unscaled products and applies the operands' power-of-two
// scale factors once per output (stored tensors are kept near 1 by the
// rescaling, so the unscaled products stay in range).
template <typename T, int NS, int NT, int SEMI>
__global__ void __launch_bounds__(256) k_absorb(const __grid_constant__ ADesc d) {
    constexpr int U = NS * NT <= 16 ? 4 : NS * NT <= 64 ? 2 : 1;
    const int64_t beta = blockIdx.y;
    T mx = 0;
    T scale = T(1);
    if (SEMI == SUM) {
        T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
        T sw = d.mxw ? pow2neg<T>(exp_of_bits(d.mxw[beta * d.mxw_bs])) : T(1);
        scale = sx * sw;
    }
    const int nod = d.nrd - d.nin_d;
    const int64_t ctiles = (d.nin + A_TILE - 1) / A_TILE;
    const int64_t ntiles = d.nouter * ctiles;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t o = tile / ctiles, c = tile - o * ctiles;
        int64_t bx = beta * d.bsx, by = beta * d.bsy, bw = beta * d.bsw;
        {
            int64_t r = o;
            for (int i = nod - 1; i >= 0; --i) {
                int64_t dg = r % d.rsz[i];
                r /= d.rsz[i];
                bx += dg * d.rsx[i];
                by += dg * d.rsy[i];
                bw += dg * d.rsw[i];
            }
        }
      for (int sub = 0; sub < A_TILE / (256 * U); ++sub) {
        int ox[U], oy[U], ow[U];
        bool on[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int ii = (int)(c * A_TILE) + sub * 256 * U + threadIdx.x + u * 256;
            on[u] = ii < d.nin;
            int r = on[u] ? ii : 0, x0 = 0, y0 = 0, w0 = 0;
            if (d.pow2r) {
                for (int i = nod; i < d.nrd; ++i) {
                    int dg = (r >> d.rsh[i]) & (d.rsz[i] - 1);
                    x0 += dg * (int)d.rsx[i];
                    y0 += dg * (int)d.rsy[i];
                    w0 += dg * (int)d.rsw[i];
                }
            } else {
                for (int i = d.nrd - 1; i >= nod; --i) {
                    int dg = r % d.rsz[i];
                    r /= d.rsz[i];
                    x0 += dg * (int)d.rsx[i];
                    y0 += dg * (int)d.rsy[i];
                    w0 += dg * (int)d.rsw[i];
                }
            }
            ox[u] = x0;
            oy[u] = y0;
            ow[u] = w0;
        }
        const T *Xb = (const T *)d.X + bx;
        const T *Wb = (const T *)d.W + bw;
        T *Yb = (T *)d.Y + by;
        T x[U][NS];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < NS; ++s)
                x[u][s] = (on[u] && s < d.ns) ? Xb[ox[u] + d.xoff[s]] : T(0);
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

template <typename T, int NS, int NT>
static void absorb_go(const ADesc &d, int semiring, cudaStream_t st) {
    int64_t tiles = d.nouter * ((d.nin + A_TILE - 1) / A_TILE);
    int64_t cap = std::max<int64_t>(1, (152LL * 16) / std::max(1, d.nbeta));
    dim3 grid((unsigned)std::max<int64_t>(1, std::min(tiles, cap)), (unsigned)d.nbeta, 1);
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

template <typename T, int NS, int NT>
__global__ void __launch_bounds__(256) k_reduce_part(const __grid_constant__ RDesc d,
                                                     int64_t chunk, int nchunks, T *part) {
    int64_t g = (int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z;
    if (g >= d.ng * d.nbeta) return;
    int64_t beta = g / d.ng, gi = g - beta * d.ng;
    int64_t ox = beta * d.bsx, oz = beta * d.bsz, oo = 0;
    group_offsets(d, gi, ox, oz, oo);
    const T *X = (const T *)d.X + ox;
    const T *Z = (const T *)d.Z + oz;
    T sx = d.mxx ? pow2neg<T>(exp_of_bits(d.mxx[beta * d.mxx_bs])) : T(1);
    T sz = d.mxz ? pow2neg<T>(exp_of_bits(d.mxz[beta * d.mxz_bs])) : T(1);
    T acc[NS][NT];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int t = 0; t < NT; ++t) acc[s][t] = 0;
    int64_t m0 = (int64_t)blockIdx.x * chunk, m1 = min(m0 + chunk, d.nm);
    constexpr int U = NS * NT <= 4 ? 4 : NS * NT <= 16 ? 2 : 1;
    for (int64_t mb = m0 + threadIdx.x; mb < m1; mb += (int64_t)blockDim.x * U) {
        T x[U][NS], z[U][NT];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int64_t m = mb + (int64_t)u * blockDim.x;
            bool on = m < m1;
            int64_t mxo = 0, mzo = 0;
            if (d.pow2m) {
#pragma unroll 4
                for (int i = 0; i < d.nmd; ++i) {
                    int64_t dg = (m >> d.msh[i]) & (int64_t)(d.msz[i] - 1);
                    mxo += dg * d.msx[i];
                    mzo += dg * d.msz2[i];
                }
            } else {
                int64_t r = m;
                for (int i = d.nmd - 1; i >= 0; --i) {
                    int64_t dg = r % d.msz[i];
                    r /= d.msz[i];
                    mxo += dg * d.msx[i];
                    mzo += dg * d.msz2[i];
                }
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) x[u][s] = (on && s < d.ns) ? X[mxo + d.xoff[s]] : T(0);
#pragma unroll
            for (int t = 0; t < NT; ++t) z[u][t] = (on && t < d.nt) ? Z[mzo + d.zoff[t]] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int t = 0; t < NT; ++t) acc[s][t] += (x[u][s] * sx) * (z[u][t] * sz);
    }
    __shared__ T red[8][NS * NT];
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
    for (int i = threadIdx.x; i < NS * NT; i += blockDim.x) {
        T v = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) v += red[q][i];
        part[(g * nchunks + blockIdx.x) * (NS * NT) + i] = v;
    }
}

template <typename T, int NS, int NT>
__global__ void __launch_bounds__(256) k_reduce_fin(const __grid_constant__ RDesc d, int nchunks,
                                                    const T *part) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t tot = d.ng * d.nbeta * NS * NT;
    bool active = idx < tot;
    int64_t beta = 0;
    double v = 0;
    if (active) {
        int64_t g = idx / (NS * NT);
        int i = (int)(idx - g * (NS * NT));
        int s = i / NT, t = i % NT;
        beta = g / d.ng;
        if (s < d.ns && t < d.nt) {
            T acc = 0;
            for (int c = 0; c < nchunks; ++c) acc += part[(g * nchunks + c) * (NS * NT) + i];
            int64_t ox = 0, oz = 0, oo = beta * d.bso;
            group_offsets(d, g - beta * d.ng, ox, oz, oo);
            ((T *)d.O)[oo + d.oso[s] + d.oto[t]] = acc;
            v = (double)acc;
        } else {
            active = false;
        }
    }
    record_max(d.mxo, beta, active, v);
}

static void reduce_shape(const RDesc &d, int64_t &chunk, int &nchunks) {
    int64_t groups = d.ng * d.nbeta;
    int64_t want = std::max<int64_t>(1, (152LL * 8) / std::max<int64_t>(1, groups));
    chunk = std::max<int64_t>(2048, (d.nm + want - 1) / want);
    nchunks = (int)((d.nm + chunk - 1) / chunk);
}

static int reduce_tile(const RDesc &d) {
    int m = std::min(8, d.ns > d.nt ? d.ns : d.nt);
    return m <= 1 ? 1 : m <= 2 ? 2 : m <= 4 ? 4 : 8;
}

#ifdef TN_STREAM_HOST_DEFS
size_t reduce_scratch_bytes(const RDesc &d, int elem_bytes) {
    int64_t chunk;
    int nchunks;
    reduce_shape(d, chunk, nchunks);
    int q = 8;
    return (size_t)(d.ng * d.nbeta * nchunks * q * q) * elem_bytes;
}
#endif

template <typename T, int Q>
static void reduce_go(const RDesc &d, void *scratch, cudaStream_t st) {
    int64_t chunk;
    int nchunks;
    reduce_shape(d, chunk, nchunks);
    int64_t groups = d.ng * d.nbeta;
    dim3 grid((unsigned)nchunks, (unsigned)std::min<int64_t>(groups, 65535),
              (unsigned)((groups + 65534) / 65535));
    k_reduce_part<T, Q, Q><<<grid, 256, 0, st>>>(d, chunk, nchunks, (T *)scratch);
    int64_t tot = groups * Q * Q;
    k_reduce_fin<T, Q, Q><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d, nchunks,
                                                                         (const T *)scratch);
}

template <typename T>
static void reduce_one(const RDesc &d, void *scratch, cudaStream_t st) {
    switch (reduce_tile(d)) {
        case 1: reduce_go<T, 1>(d, scratch, st); break;
        case 2: reduce_go<T, 2>(d, scratch, st); break;
        case 4: reduce_go<T, 4>(d, scratch, st); break;
        default: reduce_go<T, 8>(d, scratch, st); break;
    }
}

// Outputs with more than 8 x 8 (s, t) combinations run as several launches
// over 8 x 8 chunks of them (each re-reads only the operand slices it uses).
template <typename T>
void launch_reduce(const RDesc &d, void *scratch, cudaStream_t st) {
    if (d.ng * d.nbeta == 0) return;
    for (int s0 = 0; s0 < d.ns; s0 += 8)
        for (int t0 = 0; t0 < d.nt; t0 += 8) {
            RDesc c = d;
            c.ns = std::min(8, d.ns - s0);
            c.nt = std::min(8, d.nt - t0);
            for (int i = 0; i < c.ns; ++i) {
                c.xoff[i] = d.xoff[s0 + i];
                c.oso[i] = d.oso[s0 + i];
            }
            for (int i = 0; i < c.nt; ++i) {
                c.zoff[i] = d.zoff[t0 + i];
                c.oto[i] = d.oto[t0 + i];
            }
            reduce_one<T>(c, scratch, st);
        }
}

#ifdef TN_STREAM_HOST_DEFS
int reduce_launches(const RDesc &d) { return 2 * ((d.ns + 7) / 8) * ((d.nt + 7) / 8); }
#endif


}  // namespace tn

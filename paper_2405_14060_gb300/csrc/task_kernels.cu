// Task kernels around the pairwise contractions: leaf construction (factors,
// unity / evidence vectors), log Z from the root and the rescaling exponents,
// marginals from the adjoints of the unity vectors, factor marginals, MPE
// backtracking and backward sampling.
#include <cfloat>
#include <cmath>

#include "devutil.cuh"
#include "task_kernels.cuh"

namespace tn {

__device__ __forceinline__ int exp_bits(unsigned long long b) {
    if (b == 0ull) return 0;
    return (int)((b >> 52) & 0x7ffull) - 1023;
}

// ------------------------------------------------------------------ leaves
//
// Factor leaf: the model's table (optionally its logarithm, for max-plus).
// Unity leaf of variable v (Sec. MAR step 1; Sec. MPE step 1): all ones for a
// free variable; for an observed variable the indicator of its value, which
// multiplies in the slicing T_{V|E=e} of Eq. pr.  In the log domain ones are
// 0 and zeros are -inf.  Each leaf records its maximum for rescaling.
template <typename T>
__global__ void k_leaves(const LeafRec *recs, const double *tables, const int *card, int nvars,
                         const int32_t *evid, int nbeta, int log_mode, T *base,
                         unsigned long long *mx, const int *flags, const int32_t *slice_val) {
    const LeafRec r = recs[blockIdx.x];
    T *dst = base + r.dst;
    __shared__ double smax[32];
    if (r.kind == LEAF_FACTOR || r.kind == LEAF_EXTERNAL) {
        double m = log_mode ? -INFINITY : 0.0;
        for (int64_t i = threadIdx.x; i < r.size; i += blockDim.x) {
            double x;
            if (r.kind == LEAF_FACTOR) {
                int64_t off = r.src + i;
                if (r.nkd >= 0) {
                    off = r.src;
                    int64_t q = i;
                    for (int j = r.nkd - 1; j >= 0; --j) {
                        off += (q % r.ksz[j]) * r.kst[j];
                        q /= r.ksz[j];
                    }
                    for (int j = 0; j < r.nsd; ++j) off += (int64_t)slice_val[r.sidx[j]] * r.sst[j];
                }
                x = tables[off];
                bool in_log = flags && flags[0];
                if (log_mode && !in_log) x = log(x);
                else if (!log_mode && in_log) x = exp(x);
            } else {
                // external: log of a sum-product result times 2^sigma
                const T *s = (const T *)(uintptr_t)r.src;
                double sig = r.sigma ? *r.sigma : 0.0;
                double v = (double)s[i];
                x = v > 0 ? log(v) + sig * 0.69314718055994530942 : -INFINITY;
            }
            dst[i] = (T)x;
            m = fmax(m, log_mode ? (double)(T)x : x);
        }
        // the maximum: a power-of-two scale source for sum-product, the
        // max-normalisation offset (order-preserving key) for max-plus
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, s));
        if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = log_mode ? -INFINITY : 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, smax[w]);
            mx[r.mx] = log_mode ? (isfinite(t) ? okey(t) : 0ull)
                                : (unsigned long long)__double_as_longlong(t);
        }
    } else {
        int v = r.var, c = card[v];
        int nb = r.beta ? nbeta : 1;
        if (r.slice_of_var >= 0) {
            // a sliced variable's vector is the scalar u_v[slice value]
            int xs = slice_val[r.slice_of_var];
            for (int b = threadIdx.x; b < nb; b += blockDim.x) {
                int e = evid ? evid[(int64_t)b * nvars + v] : -1;
                bool one = e < 0 || e == xs;
                dst[b] = log_mode ? (one ? T(0) : T(-INFINITY)) : (one ? T(1) : T(0));
            }
            c = 1;
        } else
        for (int64_t t = threadIdx.x; t < (int64_t)nb * c; t += blockDim.x) {
            int b = (int)(t / c), x = (int)(t % c);
            int e = evid ? evid[(int64_t)b * nvars + v] : -1;
            bool one = e < 0 || e == x;
            dst[t] = log_mode ? (one ? T(0) : T(-INFINITY)) : (one ? T(1) : T(0));
        }
        if (!log_mode)
            for (int b = threadIdx.x; b < nb; b += blockDim.x)
                mx[r.mx + b] = (unsigned long long)__double_as_longlong(1.0);
    }
}

template <typename T>
void launch_leaves(const LeafRec *recs, int nrec, const double *tables, const int *card,
                   int nvars, const int32_t *evid, int nbeta, int log_mode, T *base,
                   unsigned long long *mx, const int *flags, const int32_t *slice_val,
                   cudaStream_t st) {
    if (nrec <= 0) return;
    k_leaves<T><<<nrec, 256, 0, st>>>(recs, tables, card, nvars, evid, nbeta, log_mode, base, mx,
                                      flags, slice_val);
}

// ------------------------------------------------------------ slicing

__global__ void k_slice_init(int nbeta, int64_t nm, double *M, double *S, double *A) {
    int b = blockIdx.x;
    if (threadIdx.x == 0) {
        M[b] = -INFINITY;
        S[b] = 0.0;
    }
    for (int64_t i = threadIdx.x; i < nm; i += blockDim.x) A[(int64_t)b * nm + i] = 0.0;
}

void launch_slice_init(int nbeta, int64_t nm, double *M, double *S, double *A, cudaStream_t st) {
    k_slice_init<<<nbeta, 256, 0, st>>>(nbeta, nm, M, S, A);
}

__global__ void k_slice_acc(int nbeta, const double *logz, const double *marg, int64_t nm,
                            const int32_t *slice_val, int nsl, const int32_t *sl_var,
                            const int64_t *sl_moff, const int32_t *sl_card, double *M, double *S,
                            double *A) {
    const int b = blockIdx.x;
    __shared__ double sh_scale, sh_w;
    __shared__ int sh_skip;
    if (threadIdx.x == 0) {
        double lz = logz[b];
        sh_skip = !(lz > -INFINITY);
        if (!sh_skip) {
            double m = M[b], scale = 1.0;
            if (!(m > -INFINITY) || lz > m) {
                scale = m > -INFINITY ? exp(m - lz) : 0.0;
                M[b] = lz;
                m = lz;
            }
            sh_scale = scale;
            sh_w = exp(lz - m);
            S[b] = S[b] * scale + sh_w;
        }
    }
    __syncthreads();
    if (sh_skip) return;
    const double scale = sh_scale, w = sh_w;
    double *a = A + (int64_t)b * nm;
    if (marg) {
        const double *p = marg + (int64_t)b * nm;
        for (int64_t i = threadIdx.x; i < nm; i += blockDim.x) a[i] = a[i] * scale + w * p[i];
        __syncthreads();
        for (int j = threadIdx.x; j < nsl; j += blockDim.x)
            a[sl_moff[j] + slice_val[j]] += w;
    }
    (void)sl_var;
    (void)sl_card;
}

void launch_slice_acc(int nbeta, const double *logz, const double *marg, int64_t nm,
                      const int32_t *slice_val, int nsl, const int32_t *sl_var,
                      const int64_t *sl_moff, const int32_t *sl_card, double *M, double *S,
                      double *A, cudaStream_t st) {
    k_slice_acc<<<nbeta, 256, 0, st>>>(nbeta, logz, marg, nm, slice_val, nsl, sl_var, sl_moff,
                                       sl_card, M, S, A);
}

__global__ void k_slice_fin(int nbeta, int64_t nm, const double *M, const double *S,
                            const double *A, double *logz, double *marg) {
    const int b = blockIdx.x;
    double s = S[b];
    if (threadIdx.x == 0) logz[b] = s > 0 ? M[b] + log(s) : -INFINITY;
    if (marg)
        for (int64_t i = threadIdx.x; i < nm; i += blockDim.x)
            marg[(int64_t)b * nm + i] = s > 0 ? A[(int64_t)b * nm + i] / s : NAN;
}

void launch_slice_fin(int nbeta, int64_t nm, const double *M, const double *S, const double *A,
                      double *logz, double *marg, cudaStream_t st) {
    k_slice_fin<<<nbeta, 256, 0, st>>>(nbeta, nm, M, S, A, logz, marg);
}

// ------------------------------------------------------------------- log Z
//
// log p(e_b) = ln(root_b) + ln2 * sum over every non-root tensor t of e_t(b),
// where e_t is the binary exponent removed when t was consumed.  sigma_out
// (optional) receives the log2 scale sum itself.
// One block per batch item; the exponents are integers, so the block-wide
// sum is exact in any order.
template <typename T>
__global__ void __launch_bounds__(256) k_logz(int nbeta, const T *root, int root_beta,
                                              const unsigned long long *mx, const int64_t *exps,
                                              int nexp, double *logz, double *sigma_out,
                                              int maxplus) {
    const int b = blockIdx.x;
    const double r = (double)root[root_beta ? b : 0];
    if (maxplus) {
        // log p = root + the offsets every consumer subtracted (FP64 sum in a
        // fixed order: per-thread strided sums, then a fixed tree)
        double s = 0.0;
        for (int i = threadIdx.x; i < nexp; i += blockDim.x) {
            int64_t idx = exps[2 * i], bs = exps[2 * i + 1];
            s += okey_off<double>(mx[idx + (bs ? b : 0)]);
        }
        __shared__ double dpart[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) dpart[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += dpart[w];
            logz[b] = r + t;
            if (sigma_out) sigma_out[b] = t;
        }
        return;
    }
    long long s = 0;
    for (int i = threadIdx.x; i < nexp; i += blockDim.x) {
        int64_t idx = exps[2 * i], bs = exps[2 * i + 1];
        s += exp_bits(mx[idx + (bs ? b : 0)]);
    }
    __shared__ long long part[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        if (sigma_out) sigma_out[b] = (double)t;
        logz[b] = r > 0 ? log(r) + (double)t * 0.69314718055994530942 : -INFINITY;
    }
}

template <typename T>
void launch_logz(int nbeta, const T *root, int root_beta, const unsigned long long *mx,
                 const int64_t *exps, int nexp, double *logz, double *sigma_out, int maxplus,
                 cudaStream_t st) {
    k_logz<T><<<nbeta, 256, 0, st>>>(nbeta, root, root_beta, mx, exps, nexp, logz, sigma_out,
                                     maxplus);
}

// --------------------------------------------------------------- adjoints

template <typename T>
__global__ void k_fill_one(T *p, int64_t n, unsigned long long *mx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        p[i] = T(1);
        if (mx) mx[i] = (unsigned long long)__double_as_longlong(1.0);
    }
}

template <typename T>
void launch_fill_one(T *p, int64_t n, unsigned long long *mx, cudaStream_t st) {
    k_fill_one<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, n, mx);
}

// p(v = x | e_b) = u[x] * ubar[x] / sum_y u[y] * ubar[y]: the gradient of
// p(e) with respect to the unity vector of v is p(v, e) (Sec. MAR step 3),
// and the common scale of the stored adjoint cancels in the ratio.
template <typename T>
__global__ void k_marginals(const MargRec *recs, int nvars, int nbeta, const T *fbase,
                            const T *abase, double *marg, int64_t mstride) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nvars * nbeta) return;
    int b = (int)(t / nvars), v = (int)(t % nvars);
    const MargRec r = recs[v];
    if (r.sliced) {
        double *o = marg + (int64_t)b * mstride + r.moff;
        for (int x = 0; x < r.card; ++x) o[x] = 0.0;
        return;
    }
    const T *u = fbase + r.fwd + (r.fbeta ? (int64_t)b * r.card : 0);
    const T *ub = abase + r.adj + (r.abeta ? (int64_t)b * r.card : 0);
    double s = 0;
    for (int x = 0; x < r.card; ++x) s += (double)u[x] * (double)ub[x];
    double *out = marg + (int64_t)b * mstride + r.moff;
    for (int x = 0; x < r.card; ++x)
        out[x] = s > 0 ? (double)u[x] * (double)ub[x] / s : NAN;
}

template <typename T>
void launch_marginals(const MargRec *recs, int nvars, int nbeta, const T *fbase, const T *abase,
                      double *marg, int64_t mstride, cudaStream_t st) {
    int64_t n = (int64_t)nvars * nbeta;
    k_marginals<T><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(recs, nvars, nbeta, fbase, abase,
                                                               marg, mstride);
}

// Factor marginals p(scope_f = x | e_b) = T_f[x] * Tbar_f[x] / sum, which is
// d log p(e_b) / d log T_f[x] (Thm. "Tensor network differentiation").
template <typename T>
__global__ void k_factor_grads(const GradRec *recs, int nbeta, const T *fbase, const T *abase,
                               double *grad, int64_t gstride) {
    const GradRec r = recs[blockIdx.x];
    int b = blockIdx.y;
    const T *f = fbase + r.fwd;
    const T *fb = abase + r.adj + (r.abeta ? (int64_t)b * r.size : 0);
    __shared__ double ssum[32];
    double s = 0;
    for (int64_t i = threadIdx.x; i < r.size; i += blockDim.x) s += (double)f[i] * (double)fb[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ssum[threadIdx.x >> 5] = s;
    __syncthreads();
    double tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += ssum[w];
    double *out = grad + (int64_t)b * gstride + r.goff;
    for (int64_t i = threadIdx.x; i < r.size; i += blockDim.x)
        out[i] = tot > 0 ? (double)f[i] * (double)fb[i] / tot : NAN;
}

template <typename T>
void launch_factor_grads(const GradRec *recs, int nrec, int nbeta, const T *fbase,
                         const T *abase, double *grad, int64_t gstride, cudaStream_t st) {
    if (nrec <= 0) return;
    dim3 grid((unsigned)nrec, (unsigned)nbeta);
    k_factor_grads<T><<<grid, 128, 0, st>>>(recs, nbeta, fbase, abase, grad, gstride);
}

// ---------------------------------------------------------- MPE backtrack
//
// Top-down over the internal nodes (root first): the output labels of a node
// are already assigned (root: none), so the stored argmax at that position
// gives the values of the labels maximised at the node.  This is the Boolean
// mask rule of Eq. tropical-back with the mask of each node reduced to the
// single selected entry (ties resolved to the lowest flat index when the
// maximiser was recorded).
// Record layout (int64): nC, {label, strideC} x nC, nK, {label, size} x nK,
// argmax offset, per-item output count, batch flag.
__global__ void k_backtrack(const int64_t *meta, int nnodes, const int32_t *argmax, int nbeta,
                            int nvars, int32_t *assign) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbeta) return;
    int32_t *x = assign + (int64_t)b * nvars;
    const int64_t *p = meta;
    for (int n = 0; n < nnodes; ++n) {
        int64_t nC = *p++;
        int64_t o = 0;
        for (int64_t i = 0; i < nC; ++i) {
            o += (int64_t)x[p[0]] * p[1];
            p += 2;
        }
        int64_t nK = *p++;
        const int64_t *kl = p;
        p += 2 * nK;
        int64_t aoff = p[0], per = p[1], bflag = p[2];
        p += 3;
        int64_t k = argmax[aoff + (bflag ? (int64_t)b * per : 0) + o];
        for (int64_t i = nK - 1; i >= 0; --i) {
            int64_t sz = kl[2 * i + 1];
            x[kl[2 * i]] = (int32_t)(k % sz);
            k /= sz;
        }
    }
}

void launch_backtrack(const int64_t *meta, int nnodes, const int32_t *argmax, int nbeta,
                      int nvars, int32_t *assign, cudaStream_t st) {
    k_backtrack<<<(nbeta + 63) / 64, 64, 0, st>>>(meta, nnodes, argmax, nbeta, nvars, assign);
}

// ------------------------------------------------------- backward sampling
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds of the Philox S-box with the
// multipliers 0xD2511F53, 0xCD9E8D57 and the Weyl key increments 0x9E3779B9,
// 0xBB67AE85 given in that paper.
struct P4 { uint32_t v[4]; };

__device__ __forceinline__ P4 philox4x32_10(P4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c.v[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c.v[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        P4 n;
        n.v[0] = hi1 ^ c.v[1] ^ k0;
        n.v[1] = lo1;
        n.v[2] = hi0 ^ c.v[3] ^ k1;
        n.v[3] = lo0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ double uniform01(uint64_t sample, uint32_t node, uint64_t seed) {
    P4 c;
    c.v[0] = (uint32_t)sample;
    c.v[1] = (uint32_t)(sample >> 32);
    c.v[2] = node;
    c.v[3] = 0;
    P4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t m = ((uint64_t)(r.v[0] >> 5) << 26) | (uint64_t)(r.v[1] >> 6);   // 53 bits
    return (double)m * (1.0 / 9007199254740992.0);
}

// Record layout (int64): nC, {label, sA, sB, sC} x nC, nK, {label, size, sA,
// sB} x nK, offA, offB, ktotal, cdf offset (-1: sample by direct summation).
// At a node C_Z = con({A_X, B_Y}, Z) with the sample's values s_Z already
// drawn, the eliminated labels M are drawn from A[s_Z, m] B[s_Z, m] / C[s_Z]
// (Eq. condition-prob); the stored tensors' common scales cancel.
template <typename T>
__global__ void k_sample(const int64_t *meta, int nnodes, const T *base, const double *cdf,
                         const int32_t *evid, int nvars, int64_t nsamp, uint64_t seed,
                         int8_t *out) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsamp) return;
    int8_t *x = out + s * nvars;
    for (int v = 0; v < nvars; ++v) x[v] = (int8_t)(evid && evid[v] >= 0 ? evid[v] : 0);
    const int64_t *p = meta;
    for (int n = 0; n < nnodes; ++n) {
        int64_t nC = *p++;
        int64_t oa = 0, ob = 0, oc = 0;
        for (int64_t i = 0; i < nC; ++i) {
            int64_t xv = x[p[0]];
            oa += xv * p[1];
            ob += xv * p[2];
            oc += xv * p[3];
            p += 4;
        }
        int64_t nK = *p++;
        const int64_t *kl = p;
        p += 4 * nK;
        int64_t offA = p[0], offB = p[1], K = p[2], coff = p[3];
        p += 4;
        double u = uniform01((uint64_t)s, (uint32_t)n, seed);
        int64_t pick = 0;
        if (coff >= 0) {
            const double *row = cdf + coff + oc * K;
            double r = u * row[K - 1];
            int64_t lo = 0, hi = K - 1;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (row[mid] > r) hi = mid;
                else lo = mid + 1;
            }
            pick = lo;
        } else {
            const T *A = base + offA + oa;
            const T *B = base + offB + ob;
            double tot = 0;
            for (int64_t k = 0; k < K; ++k) {
                int64_t ka = 0, kb = 0, r = k;
                for (int64_t i = nK - 1; i >= 0; --i) {
                    int64_t dg = r % kl[4 * i + 1];
                    r /= kl[4 * i + 1];
                    ka += dg * kl[4 * i + 2];
                    kb += dg * kl[4 * i + 3];
                }
                tot += (double)A[ka] * (double)B[kb];
            }
            double r0 = u * tot, c = 0;
            pick = K - 1;
            for (int64_t k = 0; k < K; ++k) {
                int64_t ka = 0, kb = 0, r = k;
                for (int64_t i = nK - 1; i >= 0; --i) {
                    int64_t dg = r % kl[4 * i + 1];
                    r /= kl[4 * i + 1];
                    ka += dg * kl[4 * i + 2];
                    kb += dg * kl[4 * i + 3];
                }
                double w = (double)A[ka] * (double)B[kb];
                c += w;
                if (r0 < c && w > 0) { pick = k; break; }
            }
        }
        for (int64_t i = nK - 1; i >= 0; --i) {
            int64_t sz = kl[4 * i + 1];
            x[kl[4 * i]] = (int8_t)(pick % sz);
            pick /= sz;
        }
    }
}

template <typename T>
void launch_sample(const int64_t *meta, int nnodes, const T *base, const double *cdf,
                   const int32_t *evid, int nvars, int64_t nsamp, uint64_t seed, int8_t *out,
                   cudaStream_t st) {
    k_sample<T><<<(unsigned)((nsamp + 127) / 128), 128, 0, st>>>(meta, nnodes, base, cdf, evid,
                                                                nvars, nsamp, seed, out);
}

// Cumulative sums cdf[o][k] = sum_{j<=k} A[o, j] B[o, j] over the summed
// labels of one node (one block per output entry), for nodes whose summed
// space is too large to scan per sample.
template <typename T>
__global__ void k_cdf_rows(const __grid_constant__ CDesc d, double *cdf) {
    int64_t o = blockIdx.x;
    int64_t oa = 0, ob = 0;
    {
        int64_t r = o;
        for (int i = d.nout - 1; i >= 0; --i) {
            int64_t dg = r % d.osz[i];
            r /= d.osz[i];
            oa += dg * d.osa[i];
            ob += dg * d.osb[i];
        }
    }
    const T *A = (const T *)d.A + oa;
    const T *B = (const T *)d.B + ob;
    int64_t K = d.ktotal;
    int nt = blockDim.x;
    int64_t per = (K + nt - 1) / nt;
    int64_t k0 = threadIdx.x * per, k1 = min(K, k0 + per);
    auto val = [&](int64_t k) {
        int64_t ka = 0, kb = 0, r = k;
        for (int i = d.nk - 1; i >= 0; --i) {
            int64_t dg = r % d.ksz[i];
            r /= d.ksz[i];
            ka += dg * d.ksa[i];
            kb += dg * d.ksb[i];
        }
        return (double)A[ka] * (double)B[kb];
    };
    double s = 0;
    for (int64_t k = k0; k < k1; ++k) s += val(k);
    __shared__ double pre[1024];
    pre[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0;
        for (int i = 0; i < nt; ++i) {
            double t = pre[i];
            pre[i] = run;
            run += t;
        }
    }
    __syncthreads();
    double run = pre[threadIdx.x];
    double *row = cdf + o * K;
    for (int64_t k = k0; k < k1; ++k) {
        run += val(k);
        row[k] = run;
    }
}

template <typename T>
void launch_cdf_rows(const CDesc &d, int64_t rows, double *cdf, cudaStream_t st) {
    k_cdf_rows<T><<<(unsigned)rows, 256, 0, st>>>(d, cdf);
}

#define INST(T)                                                                                  \
    template void launch_leaves<T>(const LeafRec *, int, const double *, const int *, int,      \
                                   const int32_t *, int, int, T *, unsigned long long *,        \
                                   const int *, const int32_t *, cudaStream_t);                 \
    template void launch_logz<T>(int, const T *, int, const unsigned long long *,              \
                                 const int64_t *, int, double *, double *, int, cudaStream_t);  \
    template void launch_fill_one<T>(T *, int64_t, unsigned long long *, cudaStream_t);         \
    template void launch_marginals<T>(const MargRec *, int, int, const T *, const T *,          \
                                      double *, int64_t, cudaStream_t);                         \
    template void launch_factor_grads<T>(const GradRec *, int, int, const T *, const T *,       \
                                         double *, int64_t, cudaStream_t);                      \
    template void launch_sample<T>(const int64_t *, int, const T *, const double *,             \
                                   const int32_t *, int, int64_t, uint64_t, int8_t *,           \
                                   cudaStream_t);                                               \
    template void launch_cdf_rows<T>(const CDesc &, int64_t, double *, cudaStream_t);
INST(float)
INST(double)

}  // namespace tn

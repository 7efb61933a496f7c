/*
 * tn_oracle.c -- plain CPU FP64 reference ("the oracle") for exact inference
 * on discrete graphical models.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path: it computes the plain definitions of the inference tasks
 * (paper Sec. "Tensor networks for probabilistic modeling"):
 *
 *   PR    p(e)       = sum_{Lambda \ E} prod_f T_f|_{E=e}           (Eq. pr)
 *   MAR   p(v=x | e) = p(v=x, e) / p(e)                             (Eq. mar-prob)
 *   MPE   argmax_{Lambda \ E} sum_f log T_f|_{E=e} and its value    (Eq. log-map)
 *   MMAP  argmax_q sum_m p(q, m, e)                                  (Eq. mmap)
 *   SAMP  draws from p(Lambda \ E | e)                               (Sec. sampling)
 *
 * by two independent routes: brute-force enumeration (tiny models) and
 * variable (bucket) elimination in FP64 with a per-table natural-log offset
 * against underflow (every model size the CPU can hold).  Marginals come from
 * a two-pass bucket-tree propagation, MPE from max-sum elimination with stored
 * argmax tables, MMAP from constrained elimination (summed variables first),
 * sampling from the stored buckets in reverse elimination order.
 *
 * Model arrays: card[nvars]; factor f has scope sv[off[f] .. off[f+1]) in
 * storage order and a row-major table (last scope variable fastest) starting
 * at tab + toff[f], where toff is the running sum of table sizes.
 * Evidence: evid[v] = observed value or -1.
 * All functions return 0 on success, a negative code on error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXS 64          /* maximum scope size of any table */
#define E_ARG (-1)
#define E_MEM (-2)
#define E_BIG (-3)
#define E_ZERO (-4)      /* p(e) = 0 */

typedef struct {
    int nv;
    int v[MAXS];         /* variable ids, storage order (last fastest) */
    int64_t st[MAXS];    /* stride of each scope variable */
    int64_t size;
    double *t;
    double lsc;          /* natural-log offset: value = t * exp(lsc) (sum mode) */
} fac_t;

/* ------------------------------------------------------------------ basics */

static const int *g_card;

static void fac_init_scope(fac_t *f, int nv, const int *vars) {
    f->nv = nv;
    int64_t s = 1;
    for (int i = nv - 1; i >= 0; --i) {
        f->v[i] = vars[i];
        f->st[i] = s;
        s *= g_card[vars[i]];
    }
    f->size = s;
    f->lsc = 0.0;
}

static int fac_alloc(fac_t *f, int nv, const int *vars) {
    if (nv > MAXS) return E_BIG;
    fac_init_scope(f, nv, vars);
    if (f->size > ((int64_t)1 << 33)) return E_BIG;
    f->t = (double *)malloc(sizeof(double) * (size_t)(f->size ? f->size : 1));
    return f->t ? 0 : E_MEM;
}

static void fac_free(fac_t *f) {
    free(f->t);
    f->t = NULL;
}

static int64_t stride_of(const fac_t *f, int var) {
    for (int i = 0; i < f->nv; ++i)
        if (f->v[i] == var) return f->st[i];
    return 0;
}

static int in_scope(const fac_t *f, int var) {
    for (int i = 0; i < f->nv; ++i)
        if (f->v[i] == var) return 1;
    return 0;
}

/* Slice factor f at the evidence: T_{V | E=e} (definition of slicing). */
static int fac_slice(const fac_t *src, const int *evid, fac_t *dst) {
    int keep[MAXS] = {0}, nk = 0;
    int64_t base = 0;
    for (int i = 0; i < src->nv; ++i) {
        int v = src->v[i];
        if (evid && evid[v] >= 0) base += (int64_t)evid[v] * src->st[i];
        else keep[nk++] = v;
    }
    int rc = fac_alloc(dst, nk, keep);
    if (rc) return rc;
    int64_t sst[MAXS];
    for (int i = 0; i < nk; ++i) sst[i] = stride_of(src, keep[i]);
    int a[MAXS] = {0};
    int64_t off = base;
    for (int64_t o = 0; o < dst->size; ++o) {
        dst->t[o] = src->t[off];
        for (int d = nk - 1; d >= 0; --d) {
            off += sst[d];
            if (++a[d] < g_card[keep[d]]) break;
            off -= sst[d] * g_card[keep[d]];
            a[d] = 0;
        }
    }
    dst->lsc = src->lsc;
    return 0;
}

/* Build the input factor list from the flat model arrays. */
static int load_factors(int nvars, const int *card, int nf, const int *off,
                        const int *sv, const double *tab, fac_t **out) {
    (void)nvars;
    g_card = card;
    fac_t *fs = (fac_t *)calloc((size_t)(nf ? nf : 1), sizeof(fac_t));
    if (!fs) return E_MEM;
    int64_t toff = 0;
    for (int f = 0; f < nf; ++f) {
        int nv = off[f + 1] - off[f];
        if (nv > MAXS) return E_BIG;
        fac_init_scope(&fs[f], nv, sv + off[f]);
        fs[f].t = (double *)(tab + toff);   /* borrowed, read-only */
        toff += fs[f].size;
    }
    *out = fs;
    return 0;
}

/* -------------------------------------------------------- brute force */

/* Enumerate every assignment of the unobserved variables (variable 0 most
 * significant); calls back with the assignment and log prod_f T_f. */
typedef void (*visit_fn)(void *ctx, const int *x, double logw);

static int brute_enumerate(int nvars, const int *card, int nf, const fac_t *fs,
                           const int *evid, visit_fn fn, void *ctx) {
    int x[1024];
    if (nvars > 1024) return E_BIG;
    int freev[1024], nfree = 0;
    double logcount = 0;
    for (int v = 0; v < nvars; ++v) {
        if (evid && evid[v] >= 0) x[v] = evid[v];
        else { x[v] = 0; freev[nfree++] = v; logcount += log2((double)card[v]); }
    }
    if (logcount > 26.5) return E_BIG;
    for (;;) {
        double lw = 0.0;
        for (int f = 0; f < nf; ++f) {
            int64_t o = 0;
            for (int i = 0; i < fs[f].nv; ++i) o += (int64_t)x[fs[f].v[i]] * fs[f].st[i];
            lw += log(fs[f].t[o]);
        }
        fn(ctx, x, lw);
        int d = nfree - 1;
        for (; d >= 0; --d) {
            int v = freev[d];
            if (++x[v] < card[v]) break;
            x[v] = 0;
        }
        if (d < 0) break;
    }
    return 0;
}

static double lse2(double a, double b) {
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + log(exp(a - m) + exp(b - m));
}

typedef struct {
    int nvars;
    const int *card;
    int64_t *moff;          /* offset of each var's marginal block */
    double logz;
    double *lmarg;          /* log-sum per (v, x) */
    double best;
    int *bestx;
    /* mmap */
    int nq;
    const int *q;
    double *lq;             /* log-sum per query configuration */
    /* joint */
    double *joint;
    const int *freev;
    int nfree;
} bctx_t;

static void visit_pr(void *c, const int *x, double lw) {
    (void)x;
    bctx_t *b = (bctx_t *)c;
    b->logz = lse2(b->logz, lw);
}

static void visit_mar(void *c, const int *x, double lw) {
    bctx_t *b = (bctx_t *)c;
    b->logz = lse2(b->logz, lw);
    for (int v = 0; v < b->nvars; ++v) {
        double *p = &b->lmarg[b->moff[v] + x[v]];
        *p = lse2(*p, lw);
    }
}

static void visit_map(void *c, const int *x, double lw) {
    bctx_t *b = (bctx_t *)c;
    if (lw > b->best) {
        b->best = lw;
        memcpy(b->bestx, x, sizeof(int) * (size_t)b->nvars);
    }
}

static void visit_mmap(void *c, const int *x, double lw) {
    bctx_t *b = (bctx_t *)c;
    int64_t idx = 0;
    for (int i = 0; i < b->nq; ++i) idx = idx * b->card[b->q[i]] + x[b->q[i]];
    b->lq[idx] = lse2(b->lq[idx], lw);
}

static void visit_joint(void *c, const int *x, double lw) {
    bctx_t *b = (bctx_t *)c;
    int64_t idx = 0;
    for (int i = 0; i < b->nfree; ++i) idx = idx * b->card[b->freev[i]] + x[b->freev[i]];
    b->joint[idx] = lw;
}

int or_brute_pr(int nvars, const int *card, int nf, const int *off, const int *sv,
                const double *tab, const int *evid, double *logz) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    bctx_t b = {0};
    b.logz = -INFINITY;
    rc = brute_enumerate(nvars, card, nf, fs, evid, visit_pr, &b);
    free(fs);
    *logz = b.logz;
    return rc;
}

/* marg: [sum card], p(v=x | e); observed variables get their one-hot. */
int or_brute_mar(int nvars, const int *card, int nf, const int *off, const int *sv,
                 const double *tab, const int *evid, double *logz, double *marg) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    bctx_t b = {0};
    b.nvars = nvars;
    b.card = card;
    b.logz = -INFINITY;
    b.moff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nvars + 1));
    int64_t tot = 0;
    for (int v = 0; v < nvars; ++v) { b.moff[v] = tot; tot += card[v]; }
    b.lmarg = (double *)malloc(sizeof(double) * (size_t)tot);
    for (int64_t i = 0; i < tot; ++i) b.lmarg[i] = -INFINITY;
    rc = brute_enumerate(nvars, card, nf, fs, evid, visit_mar, &b);
    if (!rc) {
        *logz = b.logz;
        if (b.logz == -INFINITY) rc = E_ZERO;
        else
            for (int64_t i = 0; i < tot; ++i) marg[i] = exp(b.lmarg[i] - b.logz);
    }
    free(b.moff);
    free(b.lmarg);
    free(fs);
    return rc;
}

/* MPE by enumeration; ties go to the lexicographically smallest assignment
 * (variable 0 most significant), since only a strictly better value replaces
 * the incumbent. */
int or_brute_map(int nvars, const int *card, int nf, const int *off, const int *sv,
                 const double *tab, const int *evid, int *assign, double *logp) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    bctx_t b = {0};
    b.nvars = nvars;
    b.best = -INFINITY;
    b.bestx = assign;
    for (int v = 0; v < nvars; ++v) assign[v] = evid && evid[v] >= 0 ? evid[v] : 0;
    rc = brute_enumerate(nvars, card, nf, fs, evid, visit_map, &b);
    *logp = b.best;
    free(fs);
    if (!rc && b.best == -INFINITY) rc = E_ZERO;
    return rc;
}

/* MMAP by enumeration: log sum_m p(q, m, e) for every q, then the argmax
 * (lexicographically smallest q on ties, q[0] most significant). */
int or_brute_mmap(int nvars, const int *card, int nf, const int *off, const int *sv,
                  const double *tab, const int *evid, int nq, const int *q,
                  int *assign, double *logp) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    int64_t nqc = 1;
    for (int i = 0; i < nq; ++i) nqc *= card[q[i]];
    bctx_t b = {0};
    b.card = card;
    b.nq = nq;
    b.q = q;
    b.lq = (double *)malloc(sizeof(double) * (size_t)nqc);
    for (int64_t i = 0; i < nqc; ++i) b.lq[i] = -INFINITY;
    rc = brute_enumerate(nvars, card, nf, fs, evid, visit_mmap, &b);
    if (!rc) {
        int64_t bi = 0;
        for (int64_t i = 1; i < nqc; ++i)
            if (b.lq[i] > b.lq[bi]) bi = i;
        *logp = b.lq[bi];
        for (int i = nq - 1; i >= 0; --i) {
            assign[i] = (int)(bi % card[q[i]]);
            bi /= card[q[i]];
        }
        if (*logp == -INFINITY) rc = E_ZERO;
    }
    free(b.lq);
    free(fs);
    return rc;
}

/* Normalised joint distribution over the unobserved variables, free
 * variables in increasing id order, last fastest. */
int or_brute_joint(int nvars, const int *card, int nf, const int *off, const int *sv,
                   const double *tab, const int *evid, double *joint) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    int freev[1024], nfree = 0;
    int64_t n = 1;
    for (int v = 0; v < nvars; ++v)
        if (!(evid && evid[v] >= 0)) { freev[nfree++] = v; n *= card[v]; }
    bctx_t b = {0};
    b.card = card;
    b.joint = joint;
    b.freev = freev;
    b.nfree = nfree;
    rc = brute_enumerate(nvars, card, nf, fs, evid, visit_joint, &b);
    if (!rc) {
        double lz = -INFINITY;
        for (int64_t i = 0; i < n; ++i) lz = lse2(lz, joint[i]);
        for (int64_t i = 0; i < n; ++i) joint[i] = exp(joint[i] - lz);
    }
    free(fs);
    return rc;
}

/* ------------------------------------------------------- elimination order */

/* Greedy min-fill order over the variables for which elim[v] != 0, on the
 * interaction graph of the given factors (ties: fewer neighbours, then the
 * smaller id).  Variables with elim[v] == 0 stay in the graph but are never
 * chosen.  Writes the chosen variables to order[] and returns their count. */
static int minfill(int nvars, int nf, const fac_t *fs, const unsigned char *elim,
                   int *order) {
    unsigned char *adj = (unsigned char *)calloc((size_t)nvars * nvars, 1);
    unsigned char *gone = (unsigned char *)calloc((size_t)nvars, 1);
    for (int f = 0; f < nf; ++f)
        for (int i = 0; i < fs[f].nv; ++i)
            for (int j = 0; j < fs[f].nv; ++j)
                if (i != j) adj[(size_t)fs[f].v[i] * nvars + fs[f].v[j]] = 1;
    int cnt = 0, want = 0;
    for (int v = 0; v < nvars; ++v) want += elim[v] ? 1 : 0;
    int *nb = (int *)malloc(sizeof(int) * (size_t)nvars);
    while (cnt < want) {
        int best = -1;
        long bfill = 0;
        int bdeg = 0;
        for (int v = 0; v < nvars; ++v) {
            if (!elim[v] || gone[v]) continue;
            int k = 0;
            for (int u = 0; u < nvars; ++u)
                if (!gone[u] && adj[(size_t)v * nvars + u]) nb[k++] = u;
            long fill = 0;
            for (int a = 0; a < k; ++a)
                for (int c = a + 1; c < k; ++c)
                    if (!adj[(size_t)nb[a] * nvars + nb[c]]) ++fill;
            if (best < 0 || fill < bfill || (fill == bfill && k < bdeg)) {
                best = v;
                bfill = fill;
                bdeg = k;
            }
        }
        int k = 0;
        for (int u = 0; u < nvars; ++u)
            if (!gone[u] && adj[(size_t)best * nvars + u]) nb[k++] = u;
        for (int a = 0; a < k; ++a)
            for (int c = 0; c < k; ++c)
                if (a != c) adj[(size_t)nb[a] * nvars + nb[c]] = 1;
        gone[best] = 1;
        order[cnt++] = best;
    }
    free(nb);
    free(adj);
    free(gone);
    return cnt;
}

/* ------------------------------------------------- multiply and eliminate */

enum { OP_SUM = 0, OP_MAXSUM = 1 };

static int cmp_int(const void *a, const void *b) {
    return (*(const int *)a) - (*(const int *)b);
}

/* Output scope: union of the factors' scopes minus `skip` (or minus the
 * variables in skipset[]), sorted ascending.  Returns count. */
static int union_scope(int nf, fac_t *const *fs, int skip, int *out) {
    int n = 0;
    for (int f = 0; f < nf; ++f)
        for (int i = 0; i < fs[f]->nv; ++i) {
            int v = fs[f]->v[i];
            if (v == skip) continue;
            int seen = 0;
            for (int j = 0; j < n; ++j)
                if (out[j] == v) { seen = 1; break; }
            if (!seen) out[n++] = v;
        }
    qsort(out, (size_t)n, sizeof(int), cmp_int);
    return n;
}

/*
 * g(U \ {v}) = (+)_{x_v} (x)_f f(U_f)   over the union U of the scopes.
 *   OP_SUM:    sum-product on probability tables; the result is divided by
 *              its maximum and the log of that maximum added to lsc.
 *   OP_MAXSUM: max-sum on log tables; am (if non-NULL) receives, for every
 *              output entry, the smallest maximising value of v.
 * v = -1 multiplies without eliminating.
 */
static int multiply_eliminate(int nf, fac_t *const *fs, int v, int op, fac_t *out,
                              int **am_out) {
    int us[MAXS + 1];
    int nu = union_scope(nf, fs, v, us);
    if (nu > MAXS) return E_BIG;
    int rc = fac_alloc(out, nu, us);
    if (rc) return rc;
    int cv = v >= 0 ? g_card[v] : 1;
    int *am = NULL;
    if (am_out) {
        am = (int *)malloc(sizeof(int) * (size_t)(out->size ? out->size : 1));
        if (!am) return E_MEM;
    }
    /* per factor: stride along each output dimension and along v */
    int64_t fst[32][MAXS];
    int64_t vst[32];
    if (nf > 32) return E_BIG;
    for (int f = 0; f < nf; ++f) {
        for (int d = 0; d < nu; ++d) fst[f][d] = stride_of(fs[f], us[d]);
        vst[f] = v >= 0 ? stride_of(fs[f], v) : 0;
    }
    int64_t N = out->size;
    const int *card = g_card;
#pragma omp parallel
    {
        int nth = 1, tid = 0;
#ifdef _OPENMP
        nth = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        int64_t lo = N * tid / nth, hi = N * (tid + 1) / nth;
        int a[MAXS];
        int64_t offs[32];
        int64_t rem = lo;
        for (int d = nu - 1; d >= 0; --d) {
            a[d] = (int)(rem % card[us[d]]);
            rem /= card[us[d]];
        }
        for (int f = 0; f < nf; ++f) {
            offs[f] = 0;
            for (int d = 0; d < nu; ++d) offs[f] += fst[f][d] * a[d];
        }
        for (int64_t o = lo; o < hi; ++o) {
            if (op == OP_SUM) {
                double acc = 0.0;
                for (int x = 0; x < cv; ++x) {
                    double p = 1.0;
                    for (int f = 0; f < nf; ++f) p *= fs[f]->t[offs[f] + x * vst[f]];
                    acc += p;
                }
                out->t[o] = acc;
            } else {
                double best = -INFINITY;
                int bx = 0;
                for (int x = 0; x < cv; ++x) {
                    double s = 0.0;
                    for (int f = 0; f < nf; ++f) s += fs[f]->t[offs[f] + x * vst[f]];
                    if (s > best) { best = s; bx = x; }
                }
                out->t[o] = best;
                if (am) am[o] = bx;
            }
            for (int d = nu - 1; d >= 0; --d) {
                for (int f = 0; f < nf; ++f) offs[f] += fst[f][d];
                if (++a[d] < card[us[d]]) break;
                for (int f = 0; f < nf; ++f) offs[f] -= fst[f][d] * card[us[d]];
                a[d] = 0;
            }
        }
    }
    double lsc = 0.0;
    for (int f = 0; f < nf; ++f) lsc += fs[f]->lsc;
    out->lsc = lsc;
    if (op == OP_SUM) {
        double m = 0.0;
        for (int64_t o = 0; o < N; ++o)
            if (out->t[o] > m) m = out->t[o];
        if (m > 0.0) {
            double inv = 1.0 / m;
            for (int64_t o = 0; o < N; ++o) out->t[o] *= inv;
            out->lsc += log(m);
        } else {
            out->lsc = -INFINITY;
        }
    }
    if (am_out) *am_out = am;
    return 0;
}

/* dst(W) = sum over the variables of src not in W of src, broadcast along
 * the variables of W that src lacks.  Iterates over the union scope. */
static int marginalize_onto(const fac_t *src, fac_t *dst) {
    int us[2 * MAXS], nu = 0;
    for (int i = 0; i < src->nv; ++i) us[nu++] = src->v[i];
    for (int i = 0; i < dst->nv; ++i)
        if (!in_scope(src, dst->v[i])) us[nu++] = dst->v[i];
    int64_t ss[2 * MAXS], ds[2 * MAXS];
    for (int d = 0; d < nu; ++d) {
        ss[d] = stride_of(src, us[d]);
        ds[d] = stride_of(dst, us[d]);
    }
    memset(dst->t, 0, sizeof(double) * (size_t)dst->size);
    int a[2 * MAXS] = {0};
    int64_t so = 0, dof = 0;
    for (;;) {
        dst->t[dof] += src->t[so];
        int d = nu - 1;
        for (; d >= 0; --d) {
            so += ss[d];
            dof += ds[d];
            if (++a[d] < g_card[us[d]]) break;
            so -= ss[d] * g_card[us[d]];
            dof -= ds[d] * g_card[us[d]];
            a[d] = 0;
        }
        if (d < 0) break;
    }
    return 0;
}

/* ------------------------------------------------------------ VE machinery */

typedef struct {
    int n;            /* number of buckets (eliminated variables) */
    int *var;         /* var[i]: variable of bucket i */
    int *pos;         /* pos[v]: bucket index of v, -1 if not eliminated */
    /* bucket contents: original (sliced) factors + messages */
    int *nin;         /* count of functions in bucket i */
    int **in;         /* function ids: >=0 original factor, <0: -(1+child bucket) */
    fac_t *msg;       /* msg[i]: lambda message from bucket i */
    int *parent;      /* bucket receiving msg[i], or -1 (constant) */
    int **am;         /* MAXSUM argmax tables */
} bte_t;

typedef struct {
    int nf;
    fac_t *f;         /* sliced factors (owned) */
    double lconst;    /* accumulated log constant of scope-free factors */
} sliced_t;

static int slice_all(int nvars, const int *card, int nf, const int *off, const int *sv,
                     const double *tab, const int *evid, int logdomain, sliced_t *S) {
    fac_t *fs;
    int rc = load_factors(nvars, card, nf, off, sv, tab, &fs);
    if (rc) return rc;
    S->nf = nf;
    S->f = (fac_t *)calloc((size_t)(nf ? nf : 1), sizeof(fac_t));
    S->lconst = 0.0;
    for (int f = 0; f < nf; ++f) {
        rc = fac_slice(&fs[f], evid, &S->f[f]);
        if (rc) return rc;
        if (logdomain)
            for (int64_t i = 0; i < S->f[f].size; ++i) S->f[f].t[i] = log(S->f[f].t[i]);
    }
    free(fs);
    return 0;
}

static void sliced_free(sliced_t *S) {
    for (int f = 0; f < S->nf; ++f) fac_free(&S->f[f]);
    free(S->f);
}

static fac_t *bte_fn(bte_t *B, sliced_t *S, int id) {
    return id >= 0 ? &S->f[id] : &B->msg[-(id + 1)];
}

static void bte_add(bte_t *B, int i, int id) {
    B->in[i] = (int *)realloc(B->in[i], sizeof(int) * (size_t)(B->nin[i] + 1));
    B->in[i][B->nin[i]++] = id;
}

/* Forward (upward) pass of bucket elimination along order[0..n).  Factors
 * with no eliminated variable, and messages with empty scope, go to the
 * root list (parent -1).  Returns log of the product of all root items in
 * *lroot (sum mode) or their sum (max-sum mode). */
static int bte_forward_k(int nvars, sliced_t *S, const int *order, int n, int op,
                         bte_t *B, double *lroot, int keep);

static int bte_forward(int nvars, sliced_t *S, const int *order, int n, int op,
                       bte_t *B, double *lroot) {
    return bte_forward_k(nvars, S, order, n, op, B, lroot, 1);
}

/* keep = 0 frees every message once its receiving bucket has used it;
 * keep = -1 additionally allows variables outside `order` (a partial
 * elimination): functions holding none of the ordered variables are left
 * aside and the messages over them discarded. */
static int bte_forward_k(int nvars, sliced_t *S, const int *order, int n, int op,
                         bte_t *B, double *lroot, int keep) {
    const int partial = keep < 0;
    if (partial) keep = 0;
    memset(B, 0, sizeof(*B));
    B->n = n;
    B->var = (int *)malloc(sizeof(int) * (size_t)(n ? n : 1));
    B->pos = (int *)malloc(sizeof(int) * (size_t)nvars);
    B->nin = (int *)calloc((size_t)(n ? n : 1), sizeof(int));
    B->in = (int **)calloc((size_t)(n ? n : 1), sizeof(int *));
    B->msg = (fac_t *)calloc((size_t)(n ? n : 1), sizeof(fac_t));
    B->parent = (int *)malloc(sizeof(int) * (size_t)(n ? n : 1));
    B->am = (int **)calloc((size_t)(n ? n : 1), sizeof(int *));
    for (int v = 0; v < nvars; ++v) B->pos[v] = -1;
    for (int i = 0; i < n; ++i) { B->var[i] = order[i]; B->pos[order[i]] = i; }
    double root = 0.0;
    for (int f = 0; f < S->nf; ++f) {
        int b = -1;
        for (int k = 0; k < S->f[f].nv; ++k) {
            int p = B->pos[S->f[f].v[k]];
            if (p >= 0 && (b < 0 || p < b)) b = p;
        }
        if (b >= 0) bte_add(B, b, f);
        else if (partial) continue;
        else {
            /* a factor whose variables are all kept (never eliminated) is a
             * root item only if it has no variables at all */
            if (S->f[f].nv != 0) return E_ARG;
            if (op == OP_SUM) root += log(S->f[f].t[0]) + S->f[f].lsc;
            else root += S->f[f].t[0];
        }
    }
    for (int i = 0; i < n; ++i) {
        fac_t *fl[64];
        int k = B->nin[i];
        if (k > 64) return E_BIG;
        if (k == 0) {
            /* lone variable: sum gives card, max-sum gives 0 */
            int nov[1] = {0};
            int rc = fac_alloc(&B->msg[i], 0, nov);
            if (rc) return rc;
            B->msg[i].t[0] = op == OP_SUM ? (double)g_card[B->var[i]] : 0.0;
            if (op == OP_MAXSUM) {
                B->am[i] = (int *)malloc(sizeof(int));
                B->am[i][0] = 0;
            }
        } else {
            for (int j = 0; j < k; ++j) fl[j] = bte_fn(B, S, B->in[i][j]);
            int rc = multiply_eliminate(k, fl, B->var[i], op, &B->msg[i],
                                        op == OP_MAXSUM ? &B->am[i] : NULL);
            if (rc) return rc;
            if (!keep)
                for (int j = 0; j < k; ++j)
                    if (B->in[i][j] < 0) fac_free(&B->msg[-(B->in[i][j] + 1)]);
        }
        int p = -1;
        for (int j = 0; j < B->msg[i].nv; ++j) {
            int q = B->pos[B->msg[i].v[j]];
            if (q < 0) {
                if (partial) continue;
                return E_ARG;
            }
            if (p < 0 || q < p) p = q;
        }
        B->parent[i] = p;
        if (p < 0 && partial && B->msg[i].nv > 0) {
            fac_free(&B->msg[i]);
            continue;
        }
        if (p >= 0) bte_add(B, p, -(i + 1));
        else if (op == OP_SUM) root += log(B->msg[i].t[0]) + B->msg[i].lsc;
        else root += B->msg[i].t[0];
    }
    *lroot = root;
    return 0;
}

static void bte_free(bte_t *B) {
    for (int i = 0; i < B->n; ++i) {
        fac_free(&B->msg[i]);
        free(B->in[i]);
        free(B->am[i]);
    }
    free(B->var); free(B->pos); free(B->nin); free(B->in);
    free(B->msg); free(B->parent); free(B->am);
}

static int make_order(int nvars, sliced_t *S, const int *evid, const int *order_in,
                      int *order) {
    if (order_in) {
        int n = 0;
        for (int i = 0; i < nvars && order_in[i] >= 0; ++i)
            if (!(evid && evid[order_in[i]] >= 0)) order[n++] = order_in[i];
        return n;
    }
    unsigned char *el = (unsigned char *)malloc((size_t)nvars);
    for (int v = 0; v < nvars; ++v) el[v] = !(evid && evid[v] >= 0);
    int n = minfill(nvars, S->nf, S->f, el, order);
    free(el);
    return n;
}

/* log2 of the largest table a min-fill elimination creates. */
int or_minfill_order(int nvars, const int *card, int nf, const int *off, const int *sv,
                     const double *tab, const int *evid, int *order, double *log2max) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    int n = make_order(nvars, &S, evid, NULL, order);
    for (int i = n; i < nvars; ++i) order[i] = -1;
    /* symbolic elimination to measure the largest table */
    int (*scope)[MAXS + 1] = malloc(sizeof(*scope) * (size_t)(S.nf + n + 1));
    int *alive = calloc((size_t)(S.nf + n + 1), sizeof(int));
    int cnt = 0;
    for (int f = 0; f < S.nf; ++f) {
        scope[cnt][0] = S.f[f].nv;
        for (int k = 0; k < S.f[f].nv; ++k) scope[cnt][1 + k] = S.f[f].v[k];
        alive[cnt++] = 1;
    }
    double best = 0;
    for (int i = 0; i < n; ++i) {
        int v = order[i], us[4 * MAXS], nu = 0;
        for (int f = 0; f < cnt; ++f) {
            if (!alive[f]) continue;
            int has = 0;
            for (int k = 0; k < scope[f][0]; ++k) if (scope[f][1 + k] == v) has = 1;
            if (!has) continue;
            alive[f] = 0;
            for (int k = 0; k < scope[f][0]; ++k) {
                int u = scope[f][1 + k], seen = 0;
                for (int j = 0; j < nu; ++j) if (us[j] == u) seen = 1;
                if (!seen && nu < 4 * MAXS) us[nu++] = u;
            }
        }
        double b = 0;
        for (int j = 0; j < nu; ++j) b += log2((double)card[us[j]]);
        if (b > best) best = b;
        int m = 0;
        for (int j = 0; j < nu && m < MAXS; ++j) if (us[j] != v) scope[cnt][1 + m++] = us[j];
        scope[cnt][0] = m;
        alive[cnt++] = 1;
    }
    *log2max = best;
    free(scope);
    free(alive);
    sliced_free(&S);
    return 0;
}

/* ------------------------------------------------------------------- PR */

/* log p(e) by bucket elimination.  order: NULL (min-fill) or a list of
 * variables terminated by -1 / nvars entries (observed ones are skipped). */
int or_ve_pr(int nvars, const int *card, int nf, const int *off, const int *sv,
             const double *tab, const int *evid, const int *order_in, double *logz) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int n = make_order(nvars, &S, evid, order_in, order);
    bte_t B;
    double lr;
    rc = bte_forward_k(nvars, &S, order, n, OP_SUM, &B, &lr, 0);
    if (!rc) *logz = lr;
    bte_free(&B);
    free(order);
    sliced_free(&S);
    return rc;
}

/* Bounded sample of a PR elimination: eliminate only the first `nelim`
 * variables of `order` (a full order of the unobserved variables), freeing
 * consumed messages.  work_prefix / work_full receive the sum, over the
 * buckets eliminated / over all buckets, of the entries a bucket visits
 * (product of the domain sizes of its scope), counted symbolically, so that
 * the time of the prefix scales to the time of the full elimination. */
int or_ve_pr_prefix(int nvars, const int *card, int nf, const int *off, const int *sv,
                    const double *tab, const int *evid, const int *order_in, int nelim,
                    double *work_prefix, double *work_full) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int n = make_order(nvars, &S, evid, order_in, order);
    if (nelim > n) nelim = n;
    /* symbolic work */
    {
        int (*scope)[4 * MAXS + 1] = malloc(sizeof(*scope) * (size_t)(S.nf + n + 1));
        int *alive = calloc((size_t)(S.nf + n + 1), sizeof(int));
        int cnt = 0;
        for (int f = 0; f < S.nf; ++f) {
            scope[cnt][0] = S.f[f].nv;
            for (int k = 0; k < S.f[f].nv; ++k) scope[cnt][1 + k] = S.f[f].v[k];
            alive[cnt++] = 1;
        }
        double wp = 0, wf = 0;
        for (int i = 0; i < n; ++i) {
            int v = order[i], us[4 * MAXS], nu = 0;
            for (int f = 0; f < cnt; ++f) {
                if (!alive[f]) continue;
                int has = 0;
                for (int k = 0; k < scope[f][0]; ++k) if (scope[f][1 + k] == v) has = 1;
                if (!has) continue;
                alive[f] = 0;
                for (int k = 0; k < scope[f][0]; ++k) {
                    int u = scope[f][1 + k], seen = 0;
                    for (int j = 0; j < nu; ++j) if (us[j] == u) seen = 1;
                    if (!seen && nu < 4 * MAXS) us[nu++] = u;
                }
            }
            double w = 1;
            for (int j = 0; j < nu; ++j) w *= card[us[j]];
            wf += w;
            if (i < nelim) wp += w;
            int m = 0;
            for (int j = 0; j < nu && m < 4 * MAXS; ++j) if (us[j] != v) scope[cnt][1 + m++] = us[j];
            scope[cnt][0] = m;
            alive[cnt++] = 1;
        }
        *work_prefix = wp;
        *work_full = wf;
        free(scope);
        free(alive);
    }
    bte_t B;
    double lr;
    rc = bte_forward_k(nvars, &S, order, nelim, OP_SUM, &B, &lr, -1);
    bte_free(&B);
    free(order);
    sliced_free(&S);
    return rc;
}

/* ------------------------------------------------------------------ MAR */

/* Two-pass propagation on the bucket tree.  The downward message from
 * bucket p to child c is the sum, over the variables of bucket p's functions
 * that are not in msg[c]'s scope, of the product of p's own factors, the
 * messages of p's other children and p's own downward message.  The belief
 * of bucket i is the product of its functions and its downward message; the
 * marginal of var[i] sums every other variable out of it. */
int or_ve_mar(int nvars, const int *card, int nf, const int *off, const int *sv,
              const double *tab, const int *evid, double *logz, double *marg) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int n = make_order(nvars, &S, evid, NULL, order);
    bte_t B;
    double lr;
    rc = bte_forward(nvars, &S, order, n, OP_SUM, &B, &lr);
    if (rc) goto done;
    *logz = lr;
    if (lr == -INFINITY) { rc = E_ZERO; goto done; }
    {
        fac_t *down = (fac_t *)calloc((size_t)(n ? n : 1), sizeof(fac_t));
        int *has_down = (int *)calloc((size_t)(n ? n : 1), sizeof(int));
        int64_t *moff = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvars);
        int64_t tot = 0;
        for (int v = 0; v < nvars; ++v) { moff[v] = tot; tot += card[v]; }
        for (int v = 0; v < nvars; ++v)
            if (evid && evid[v] >= 0)
                for (int x = 0; x < card[v]; ++x) marg[moff[v] + x] = x == evid[v];
        for (int i = n - 1; i >= 0; --i) {
            /* marginal of var[i] from bucket i's belief */
            fac_t *fl[66];
            int k = 0;
            for (int j = 0; j < B.nin[i]; ++j) fl[k++] = bte_fn(&B, &S, B.in[i][j]);
            if (has_down[i]) fl[k++] = &down[i];
            int v = B.var[i];
            if (k == 0) {
                for (int x = 0; x < card[v]; ++x) marg[moff[v] + x] = 1.0 / card[v];
            } else {
                fac_t bel;
                rc = multiply_eliminate(k, fl, -1, OP_SUM, &bel, NULL);
                if (rc) goto done;
                int64_t st = stride_of(&bel, v);
                double *acc = (double *)calloc((size_t)card[v], sizeof(double));
                for (int64_t o = 0; o < bel.size; ++o) acc[(o / st) % card[v]] += bel.t[o];
                double s = 0;
                for (int x = 0; x < card[v]; ++x) s += acc[x];
                for (int x = 0; x < card[v]; ++x) marg[moff[v] + x] = acc[x] / s;
                free(acc);
                fac_free(&bel);
            }
            /* downward messages to the children of bucket i */
            for (int j = 0; j < B.nin[i]; ++j) {
                int id = B.in[i][j];
                if (id >= 0) continue;
                int c = -(id + 1);
                fac_t *gl[66];
                int g = 0;
                for (int jj = 0; jj < B.nin[i]; ++jj)
                    if (jj != j) gl[g++] = bte_fn(&B, &S, B.in[i][jj]);
                if (has_down[i]) gl[g++] = &down[i];
                /* product over bucket i's scope, then sum out everything not
                 * in msg[c]'s scope */
                fac_t prod;
                if (g == 0) {
                    int nov[1] = {0};
                    rc = fac_alloc(&prod, 0, nov);
                    if (rc) goto done;
                    prod.t[0] = 1.0;
                } else {
                    rc = multiply_eliminate(g, gl, -1, OP_SUM, &prod, NULL);
                    if (rc) goto done;
                }
                fac_t *mc = &B.msg[c];
                rc = fac_alloc(&down[c], mc->nv, mc->v);
                if (rc) goto done;
                marginalize_onto(&prod, &down[c]);
                double m = 0;
                for (int64_t o = 0; o < down[c].size; ++o) if (down[c].t[o] > m) m = down[c].t[o];
                if (m > 0) for (int64_t o = 0; o < down[c].size; ++o) down[c].t[o] /= m;
                down[c].lsc = 0.0;   /* marginals are normalised: scale is irrelevant */
                has_down[c] = 1;
                fac_free(&prod);
            }
            if (has_down[i]) fac_free(&down[i]);
        }
        free(down);
        free(has_down);
        free(moff);
    }
done:
    bte_free(&B);
    free(order);
    sliced_free(&S);
    return rc;
}

/* ------------------------------------------------------------------ MPE */

/* Max-sum bucket elimination on log tables, then decoding in reverse
 * elimination order: the argmax table of bucket i, read at the already
 * decoded values of its message's scope, gives var[i]. */
static int decode_buckets(bte_t *B, int *x) {
    for (int i = B->n - 1; i >= 0; --i) {
        fac_t *m = &B->msg[i];
        int64_t o = 0;
        for (int d = 0; d < m->nv; ++d) o += (int64_t)x[m->v[d]] * m->st[d];
        x[B->var[i]] = B->am[i][o];
    }
    return 0;
}

int or_ve_map(int nvars, const int *card, int nf, const int *off, const int *sv,
              const double *tab, const int *evid, const int *order_in, int *assign,
              double *logp) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 1, &S);
    if (rc) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int n = make_order(nvars, &S, evid, order_in, order);
    bte_t B;
    double lr;
    rc = bte_forward(nvars, &S, order, n, OP_MAXSUM, &B, &lr);
    if (!rc) {
        for (int v = 0; v < nvars; ++v) assign[v] = evid && evid[v] >= 0 ? evid[v] : 0;
        decode_buckets(&B, assign);
        *logp = lr;
        if (lr == -INFINITY) rc = E_ZERO;
    }
    bte_free(&B);
    free(order);
    sliced_free(&S);
    return rc;
}

/* Log of prod_f T_f at a full assignment (FP64). */
double or_log_weight(int nvars, const int *card, int nf, const int *off, const int *sv,
                     const double *tab, const int *x) {
    fac_t *fs;
    if (load_factors(nvars, card, nf, off, sv, tab, &fs)) return NAN;
    double lw = 0;
    for (int f = 0; f < nf; ++f) {
        int64_t o = 0;
        for (int i = 0; i < fs[f].nv; ++i) o += (int64_t)x[fs[f].v[i]] * fs[f].st[i];
        lw += log(fs[f].t[o]);
    }
    free(fs);
    return lw;
}

/* ----------------------------------------------------------------- MMAP */

/* Constrained elimination: the summed variables (neither observed nor
 * queried) are eliminated first by sum-product, then the query variables by
 * max-sum on the logs of what remains; the query assignment is decoded from
 * the max-sum buckets. */
int or_ve_mmap(int nvars, const int *card, int nf, const int *off, const int *sv,
               const double *tab, const int *evid, int nq, const int *q,
               int *assign, double *logp) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    unsigned char *isq = (unsigned char *)calloc((size_t)nvars, 1);
    for (int i = 0; i < nq; ++i) isq[q[i]] = 1;
    unsigned char *el = (unsigned char *)malloc((size_t)nvars);
    for (int v = 0; v < nvars; ++v) el[v] = !(evid && evid[v] >= 0) && !isq[v];
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int ns = minfill(nvars, S.nf, S.f, el, order);
    /* phase 1: sum out the summed variables; functions left over after the
     * phase (those whose scope holds only query variables) form the phase-2
     * factor set */
    bte_t B;
    memset(&B, 0, sizeof(B));
    {
        /* run the forward pass over the summed variables only; items whose
         * remaining scope contains no summed variable are collected */
        B.n = ns;
        B.var = order;
        B.pos = (int *)malloc(sizeof(int) * (size_t)nvars);
        for (int v = 0; v < nvars; ++v) B.pos[v] = -1;
        for (int i = 0; i < ns; ++i) B.pos[order[i]] = i;
        B.nin = (int *)calloc((size_t)(ns ? ns : 1), sizeof(int));
        B.in = (int **)calloc((size_t)(ns ? ns : 1), sizeof(int *));
        B.msg = (fac_t *)calloc((size_t)(ns ? ns : 1), sizeof(fac_t));
        B.parent = (int *)malloc(sizeof(int) * (size_t)(ns ? ns : 1));
        B.am = (int **)calloc((size_t)(ns ? ns : 1), sizeof(int *));
    }
    sliced_t P2;
    P2.nf = 0;
    P2.f = (fac_t *)calloc((size_t)(S.nf + ns + 1), sizeof(fac_t));
    P2.lconst = 0;
    double lconst = 0.0;
    int *leftover = (int *)malloc(sizeof(int) * (size_t)(S.nf + ns + 1));
    int nleft = 0;
    for (int f = 0; f < S.nf; ++f) {
        int b = -1;
        for (int k = 0; k < S.f[f].nv; ++k) {
            int p = B.pos[S.f[f].v[k]];
            if (p >= 0 && (b < 0 || p < b)) b = p;
        }
        if (b >= 0) bte_add(&B, b, f);
        else leftover[nleft++] = f;
    }
    for (int i = 0; i < ns; ++i) {
        fac_t *fl[64];
        int k = B.nin[i];
        if (k == 0) {
            int nov[1] = {0};
            rc = fac_alloc(&B.msg[i], 0, nov);
            if (rc) goto done;
            B.msg[i].t[0] = card[B.var[i]];
        } else {
            if (k > 64) { rc = E_BIG; goto done; }
            for (int j = 0; j < k; ++j) fl[j] = bte_fn(&B, &S, B.in[i][j]);
            rc = multiply_eliminate(k, fl, B.var[i], OP_SUM, &B.msg[i], NULL);
            if (rc) goto done;
        }
        int p = -1;
        for (int j = 0; j < B.msg[i].nv; ++j) {
            int qq = B.pos[B.msg[i].v[j]];
            if (qq >= 0 && (p < 0 || qq < p)) p = qq;
        }
        B.parent[i] = p;
        if (p >= 0) bte_add(&B, p, -(i + 1));
        else leftover[nleft++] = -(i + 1);
    }
    /* phase 2: logs of the leftover functions (value * exp(lsc)) */
    for (int j = 0; j < nleft; ++j) {
        fac_t *src = bte_fn(&B, &S, leftover[j]);
        if (src->nv == 0) {
            lconst += log(src->t[0]) + src->lsc;
            continue;
        }
        fac_t *dst = &P2.f[P2.nf++];
        rc = fac_alloc(dst, src->nv, src->v);
        if (rc) goto done;
        for (int64_t i = 0; i < src->size; ++i) dst->t[i] = log(src->t[i]) + src->lsc;
    }
    {
        unsigned char *elq = (unsigned char *)calloc((size_t)nvars, 1);
        for (int i = 0; i < nq; ++i) elq[q[i]] = 1;
        int *qorder = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
        int nqo = minfill(nvars, P2.nf, P2.f, elq, qorder);
        bte_t B2;
        double lr;
        rc = bte_forward(nvars, &P2, qorder, nqo, OP_MAXSUM, &B2, &lr);
        if (!rc) {
            int *x = (int *)calloc((size_t)nvars, sizeof(int));
            decode_buckets(&B2, x);
            for (int i = 0; i < nq; ++i) assign[i] = x[q[i]];
            *logp = lr + lconst;
            if (*logp == -INFINITY) rc = E_ZERO;
            free(x);
        }
        bte_free(&B2);
        free(qorder);
        free(elq);
    }
done:
    for (int i = 0; i < ns; ++i) { fac_free(&B.msg[i]); free(B.in[i]); }
    free(B.pos); free(B.nin); free(B.in); free(B.msg); free(B.parent); free(B.am);
    for (int f = 0; f < P2.nf; ++f) fac_free(&P2.f[f]);
    free(P2.f);
    free(leftover);
    free(order);
    free(el);
    free(isq);
    sliced_free(&S);
    return rc;
}

/* ------------------------------------------------------------- sampling */

/* Exact samples from p(Lambda \ E | e): bucket elimination keeps every
 * message; then, in reverse elimination order, each variable is drawn from
 * the product of its bucket's functions evaluated at the values already
 * drawn (all other variables of those functions are eliminated later).
 * u: n * (number of free variables) uniforms in [0,1), consumed in reverse
 * elimination order per sample.  samples: [n][nvars] (observed = evidence). */
int or_ve_sample(int nvars, const int *card, int nf, const int *off, const int *sv,
                 const double *tab, const int *evid, int64_t n, const double *u,
                 int8_t *samples) {
    sliced_t S;
    int rc = slice_all(nvars, card, nf, off, sv, tab, evid, 0, &S);
    if (rc) return rc;
    int *order = (int *)malloc(sizeof(int) * (size_t)(nvars + 1));
    int nb = make_order(nvars, &S, evid, NULL, order);
    bte_t B;
    double lr;
    rc = bte_forward(nvars, &S, order, nb, OP_SUM, &B, &lr);
    if (!rc && lr == -INFINITY) rc = E_ZERO;
    if (!rc) {
        int x[1024];
        double w[64];
        for (int64_t s = 0; s < n; ++s) {
            for (int v = 0; v < nvars; ++v) x[v] = evid && evid[v] >= 0 ? evid[v] : 0;
            for (int i = nb - 1; i >= 0; --i) {
                int v = B.var[i];
                double tot = 0;
                for (int xv = 0; xv < card[v]; ++xv) {
                    x[v] = xv;
                    double p = 1.0;
                    for (int j = 0; j < B.nin[i]; ++j) {
                        fac_t *f = bte_fn(&B, &S, B.in[i][j]);
                        int64_t o = 0;
                        for (int d = 0; d < f->nv; ++d) o += (int64_t)x[f->v[d]] * f->st[d];
                        p *= f->t[o];
                    }
                    w[xv] = p;
                    tot += p;
                }
                double r = u[s * nb + (nb - 1 - i)] * tot, c = 0;
                int pick = card[v] - 1;
                for (int xv = 0; xv < card[v]; ++xv) {
                    c += w[xv];
                    if (r < c) { pick = xv; break; }
                }
                x[v] = pick;
            }
            for (int v = 0; v < nvars; ++v) samples[s * nvars + v] = (int8_t)x[v];
        }
    }
    bte_free(&B);
    free(order);
    sliced_free(&S);
    return rc;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by later calls (timing single-threaded and on all cores). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

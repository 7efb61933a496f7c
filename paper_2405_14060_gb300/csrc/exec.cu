// Executor and C ABI of libtn.
//
// A task (PR, MAR, MPE, sampling) on a model becomes a Program: the plan of
// the contraction tree (labels, layouts, summed labels per node), one device
// arena holding every tensor the task needs, one buffer of per-item maxima
// for the power-of-two rescaling, and the list of kernel launches.  The
// launches are captured once into a CUDA graph and replayed on every call, so
// a call costs one graph launch plus the copies of its inputs and outputs.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <random>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "bgemm.cuh"
#include "gemm.cuh"
#include "kernels.cuh"
#include "micro.cuh"
#include "model.h"
#include "stream.cuh"
#include "task_kernels.cuh"
#include "tn.h"
#include "tn_internal.h"

using namespace tn;

static thread_local std::string g_err;

static tn_status fail(tn_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            if (e_ == cudaErrorMemoryAllocation) cudaGetLastError();                      \
            return fail(e_ == cudaErrorMemoryAllocation ? TN_E_OOM : TN_E_CUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
        }                                                                                 \
    } while (0)

namespace {

struct Slot {
    int64_t off = -1;     // element offset in the arena
    int64_t per = 0;      // entries per item
    int64_t elems = 0;    // entries in total
    bool beta = false;
    int64_t mx = -1;      // first maximum slot
};

// First-fit offset allocator with coalescing (plan time only).
struct OffsetAlloc {
    std::map<int64_t, int64_t> freel;   // offset -> length
    int64_t top = 0;
    static int64_t round(int64_t n) { return (n + 63) & ~(int64_t)63; }
    int64_t alloc(int64_t n) {
        n = round(std::max<int64_t>(n, 1));
        for (auto it = freel.begin(); it != freel.end(); ++it)
            if (it->second >= n) {
                int64_t off = it->first, len = it->second;
                freel.erase(it);
                if (len > n) freel[off + n] = len - n;
                return off;
            }
        int64_t off = top;
        top += n;
        return off;
    }
    void release(int64_t off, int64_t n) {
        n = round(std::max<int64_t>(n, 1));
        auto it = freel.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != freel.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            freel.erase(nx);
        }
        if (it != freel.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                freel.erase(it);
            }
        }
    }
};

struct DevMem {
    std::vector<void *> ptrs;
    template <typename T>
    cudaError_t alloc(T **p, size_t bytes) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(bytes, 256));
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
    ~DevMem() {
        for (void *p : ptrs) cudaFree(p);
    }
};

enum Kind { K_PR = 0, K_MAR = 1, K_MAP = 2, K_SAMPLE = 3, K_SUMNET = 4, K_MAXNET = 5 };

// Kernel classes for profiling.
enum Cls { C_SMALL = 0, C_STREAM = 1, C_SPLITK = 2, C_TCGEMM = 3, C_SIMTGEMM = 4, C_PREP = 5,
           C_GENERIC = 6, C_BGEMM = 7, C_RECOMP = 8, C_NCLS = 9 };

struct GemmOp {
    PDesc px, py, post;
    std::vector<int32_t> tpx, tpy, tpost;   // tiled-permutation tables (host copies)
    bool has_post = false;
    bool direct = false;
    bool x_in_place = false;   // X already in GEMM form: read in place, its scale in the epilogue
    bool tc = false;
    GDesc g;
    double prep_bytes = 0, post_bytes = 0;
};

struct Step {
    int kind = 0;          // 0: strided contraction, 1: GEMM form, 2: absorb, 3: reduce,
                           // 4: batched strided GEMM
    int semiring = 0;
    CDesc d;
    GemmOp g;
    ADesc ad;
    RDesc rd;
    BDesc bd;
    std::vector<int32_t> btab;     // offset tables of a batched strided GEMM (host copy)
    double flops = 0, bytes = 0;   // algorithmic: 2 * multiply-adds; operands + result once
    const char *why = "";          // why a strided contraction did not stream (plan trace)
    int node = -1;                 // the tensor this step writes: fwd[node] or adj[node]
    bool adjoint = false;
    bool recompute = false;        // re-runs a dropped forward step before its use
    int lane = 0;                  // stream of the step inside the program's graph
    std::vector<int> waits;        // events (other lanes' results) to wait for first
    int rec = -1;                  // event to record after the step (-1: none)
};

// Launch-shape choices of a program: fixed defaults, or the fastest of a
// few candidates timed by the autotuner on the program's first use.
struct Tune {
    int max_lanes = 4;     // streams of the captured graph (1: every step in order)
    int absorb_bps = 0;    // blocks per SM of the streaming absorb kernels (0: default)
    bool tuned = false;
};

struct Program {
    int kind = 0, dtype = 0, esz = 8, nbeta = 1;
    Tune tune;
    int64_t keep_all_elems = 0;    // arena entries when every forward tensor is kept
    bool grads = false;
    Plan plan;
    std::vector<Slot> fwd, adj;
    std::vector<char> adj_beta, need_adj;
    // checkpointing (MAR under a memory budget): forward tensors not kept
    // after their parent's forward step, recomputed into rec_off[] by the
    // backward pass just before the parent's adjoint steps read them
    std::vector<char> drop;
    std::vector<int64_t> rec_off;
    int ndrop = 0;
    int64_t nmx = 0;
    DevMem mem;
    char *arena = nullptr;
    int64_t arena_elems = 0;
    unsigned long long *mx = nullptr;
    int32_t *am = nullptr;
    std::vector<int64_t> am_off;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    unsigned int *rcnt = nullptr;   // reduce steps' per-group completion counters
    int64_t nrcnt = 0;
    LeafRec *d_leaf = nullptr;
    int nleafrec = 0;
    int64_t *d_exps = nullptr;
    int nexps = 0;
    MargRec *d_margrec = nullptr;
    GradRec *d_gradrec = nullptr;
    int ngrad = 0;
    int64_t *d_meta = nullptr;
    int nmeta = 0;
    double *cdf = nullptr;
    std::vector<std::pair<CDesc, int64_t>> cdf_nodes;
    int32_t *d_evid = nullptr;
    int32_t *d_slice_val = nullptr;     // values of the sliced variables for this run
    double *d_logz = nullptr, *d_sigma = nullptr, *d_marg = nullptr, *d_grad = nullptr;
    int32_t *d_assign = nullptr;
    int *d_card = nullptr;
    std::vector<CDesc> fdesc;      // generic descriptor of every forward node
    std::vector<Step> fsteps, bsteps;
    std::vector<char> micro;                       // node runs inside a micro subtree
    std::vector<MicroDesc> mf, mb;                 // forward / backward micro lists
    std::vector<int32_t> mf_beg, mb_beg;           // per subtree start index
    MicroDesc *d_mf = nullptr, *d_mb = nullptr;
    int32_t *d_mf_beg = nullptr, *d_mb_beg = nullptr;
    char *wsX = nullptr, *wsY = nullptr, *wsD = nullptr;
    int gemm_type = 1;
    std::vector<LeafRec> leafrec;   // host copy (external sources patched per call)
    cudaGraph_t graph = nullptr;       // the captured graph (kept for multi-model launches)
    cudaGraphExec_t gexec = nullptr;
    int launches = 0;
    int64_t marg_stride = 0, grad_stride = 0;
    // independent subtrees on separate streams (lanes) of the captured graph
    int nlanes = 1;
    std::vector<int> lane;                     // per tree node
    std::vector<void *> lscratch;              // per lane: reduce / split-K scratch
    std::vector<unsigned int *> lrcnt;         // per lane: reduce completion counters
    std::vector<cudaEvent_t> ev;               // 2 NN + 2 + nlanes events (capture only)
    std::vector<int> mlane_beg;                // micro subtrees of lane l: [beg[l], beg[l+1])
    ~Program() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : ev) cudaEventDestroy(e);
    }
};

}  // namespace

// The programs of the last MMAP call (its query / evidence pattern and
// precision): a call with the same pattern replays them with new values.
struct MmapCache {
    std::vector<int8_t> key;   // per variable: 0 summed, 1 queried, 2 observed; then dtype
    std::vector<std::unique_ptr<Program>> groups;
    std::unique_ptr<Program> top;
    double lconst = 0;
};

struct tn_model {
    ModelData md;
    Tree tree;
    bool has_tree = false;
    std::vector<int> slice_vars;
    // slice combination buffers (device): running max / sum / weighted marginals
    double *d_sM = nullptr, *d_sS = nullptr, *d_sA = nullptr;
    int64_t s_cap_b = 0, s_cap_m = 0;
    int32_t *d_sl_var = nullptr, *d_sl_card = nullptr, *d_sl_tab = nullptr;
    int64_t *d_sl_moff = nullptr;
    double *d_tables = nullptr;
    int *d_flags = nullptr;            // [0]: tables hold logarithms
    int *d_err = nullptr;              // set by a device-side wait that gave up
    bool tables_overridden = false;
    int device = -1;
    cudaStream_t stream = nullptr;
    std::vector<cudaStream_t> lanes;   // extra streams that graph capture forks onto
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<Program>> progs;
    std::map<std::tuple<int, int, int, int>, Tune> tuned;   // autotuner choices per program key
    std::unique_ptr<MmapCache> mmap;
    double last_ms = 0;
    int64_t last_launches = 0;
    ~tn_model() {
        progs.clear();
        mmap.reset();
        for (void *p : {(void *)d_sM, (void *)d_sS, (void *)d_sA, (void *)d_sl_var,
                        (void *)d_sl_card, (void *)d_sl_tab, (void *)d_sl_moff})
            if (p) cudaFree(p);
        if (d_tables) cudaFree(d_tables);
        if (d_flags) cudaFree(d_flags);
        if (d_err) cudaFree(d_err);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (auto l : lanes) cudaStreamDestroy(l);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

// The model's network: factor leaves, then one unity / evidence vector per
// variable.  Sliced variables are removed from every leaf (their values are
// fixed per slice).
Net model_net(const ModelData &md, bool batched, const std::vector<int> &sliced = {}) {
    Net n;
    n.card = md.card;
    std::vector<char> sl(md.nvars, 0);
    for (int v : sliced) sl[v] = 1;
    for (int f = 0; f < md.nfactors; ++f) {
        Labels l;
        for (int v : md.scope[f])
            if (!sl[v]) l.push_back(v);
        n.leaf.push_back(l);
        n.leaf_beta.push_back(0);
    }
    for (int v = 0; v < md.nvars; ++v) {
        n.leaf.push_back(sl[v] ? Labels{} : Labels{v});
        n.leaf_beta.push_back(batched ? 1 : 0);
    }
    return n;
}

std::vector<int64_t> strides_of(const std::vector<int> &card, const Labels &l) {
    std::vector<int64_t> s(l.size());
    int64_t acc = 1;
    for (int i = (int)l.size() - 1; i >= 0; --i) {
        s[i] = acc;
        acc *= card[l[i]];
    }
    return s;
}

int64_t stride_in(const std::vector<int> &card, const Labels &l, int v) {
    int64_t acc = 1;
    for (int i = (int)l.size() - 1; i >= 0; --i) {
        if (l[i] == v) return acc;
        acc *= card[l[i]];
    }
    return -1;
}

// Descriptor of C = (+)_K A (x) B with C's labels in the given order and the
// summed labels in `korder` (default: A's labels not in C in A's order, then
// B's labels in neither, in B's order).
std::string make_desc(const std::vector<int> &card, const Labels &la, bool ba, int64_t pera,
                      const void *pA, const unsigned long long *mxa, const Labels &lb, bool bb,
                      int64_t perb, const void *pB, const unsigned long long *mxb,
                      const Labels &lc, bool bc, void *pC, unsigned long long *mxc,
                      const Labels *korder, int nbeta, int32_t *argmax, CDesc &d) {
    std::memset(&d, 0, sizeof(d));
    if ((ba || bb) && !bc) return "batch label cannot be summed";
    std::set<int> sc(lc.begin(), lc.end()), sa(la.begin(), la.end()), sb(lb.begin(), lb.end());
    Labels ks;
    if (korder) ks = *korder;
    else {
        for (int v : la)
            if (!sc.count(v)) ks.push_back(v);
        for (int v : lb)
            if (!sc.count(v) && !sa.count(v)) ks.push_back(v);
    }
    struct Dim { int64_t sz, sa, sb; };
    auto build = [&](const Labels &L, std::vector<Dim> &out) {
        std::vector<Dim> raw;
        for (int v : L) {
            if (card[v] == 1) continue;
            int64_t a = sa.count(v) ? stride_in(card, la, v) : 0;
            int64_t b = sb.count(v) ? stride_in(card, lb, v) : 0;
            raw.push_back({card[v], a, b});
        }
        out.clear();
        for (auto &x : raw) {
            if (!out.empty()) {
                Dim &c = out.back();
                if (c.sa == x.sa * x.sz && c.sb == x.sb * x.sz && c.sz * x.sz < (1LL << 31)) {
                    c.sz *= x.sz;
                    c.sa = x.sa;
                    c.sb = x.sb;
                    continue;
                }
            }
            out.push_back(x);
        }
    };
    std::vector<Dim> od, kd;
    build(lc, od);
    build(ks, kd);
    if ((int)od.size() > MAXD || (int)kd.size() > MAXD) return "contraction has too many dimensions";
    d.nout = (int)od.size();
    d.nk = (int)kd.size();
    d.nout_total = 1;
    d.ktotal = 1;
    bool p2 = true;
    for (auto &x : od) { d.nout_total *= x.sz; p2 = p2 && (x.sz & (x.sz - 1)) == 0; }
    for (auto &x : kd) { d.ktotal *= x.sz; p2 = p2 && (x.sz & (x.sz - 1)) == 0; }
    d.pow2 = p2 ? 1 : 0;
    int sh = 0;
    for (int i = d.nout - 1; i >= 0; --i) {
        d.osz[i] = (int32_t)od[i].sz;
        d.osa[i] = od[i].sa;
        d.osb[i] = od[i].sb;
        d.osh[i] = sh;
        if (p2) sh += __builtin_ctzll((unsigned long long)od[i].sz);
    }
    sh = 0;
    for (int i = d.nk - 1; i >= 0; --i) {
        d.ksz[i] = (int32_t)kd[i].sz;
        d.ksa[i] = kd[i].sa;
        d.ksb[i] = kd[i].sb;
        d.ksh[i] = sh;
        if (p2) sh += __builtin_ctzll((unsigned long long)kd[i].sz);
    }
    d.nbeta = bc ? nbeta : 1;
    d.bsa = (bc && ba) ? pera : 0;
    d.bsb = (bc && bb) ? perb : 0;
    d.A = pA;
    d.B = pB;
    d.C = pC;
    d.mxa = mxa;
    d.mxb = mxb;
    d.mxa_bs = ba ? 1 : 0;
    d.mxb_bs = bb ? 1 : 0;
    d.mxc = mxc;
    d.argmax = argmax;
    return "";
}

int64_t elem_bytes(int dtype) { return dtype == 0 ? 8 : 4; }

struct Opnd {
    const Labels *lab;
    bool beta;
    int64_t per;
    const void *ptr;
    const unsigned long long *mx;
};

struct PDim { int64_t sz, sin, sout; bool beta; };

// Fill a PDesc from logical dims (slowest first), fusing neighbours whose
// input and output strides are both contiguous.
static std::string fill_pdesc(std::vector<PDim> dims, PDesc &p) {
    std::vector<PDim> f;
    for (auto &x : dims) {
        if (x.sz == 1 && !x.beta) continue;
        if (!f.empty() && !f.back().beta && !x.beta && f.back().sin == x.sin * x.sz &&
            f.back().sout == x.sout * x.sz && f.back().sz * x.sz < (1LL << 31)) {
            f.back().sz *= x.sz;
            f.back().sin = x.sin;
            f.back().sout = x.sout;
            continue;
        }
        f.push_back(x);
    }
    if ((int)f.size() > MAXD) return "permutation has too many dimensions";
    p.nd = (int)f.size();
    p.total = 1;
    p.beta_dim = -1;
    bool p2 = true;
    for (auto &x : f) {
        p.total *= x.sz;
        p2 = p2 && (x.sz & (x.sz - 1)) == 0;
    }
    p.pow2 = p2;
    int sh = 0;
    for (int i = p.nd - 1; i >= 0; --i) {
        p.sz[i] = (int32_t)f[i].sz;
        p.sin[i] = f[i].sin;
        p.sout[i] = f[i].sout;
        p.sh[i] = sh;
        if (f[i].beta) p.beta_dim = i;
        if (p2) sh += __builtin_ctzll((unsigned long long)f[i].sz);
    }
    return "";
}

// One contraction in GEMM form: D[b][r][c] = sum_k X[b][r][k] Y[b][c][k] with
// the batch label placed in the batch group if both operands carry it, else
// in the rows (X) or columns (Y).  X and Y are prepared into workspaces in
// the GEMM input type (per-item scaled); D goes straight into the output
// tensor when its layout is [batch][rows][cols], else through a workspace
// and a scatter that records the output's per-item maxima.
static std::string make_gemm_op(const std::vector<int> &card, int nbeta, int store_t, int gemm_t,
                                const Opnd &X, const Opnd &Y, const Labels &bt,
                                const Labels &rows, const Labels &cols, const Labels &red,
                                const Labels &out_lab, bool out_beta, void *out_ptr,
                                unsigned long long *out_mx, GemmOp &op, size_t &nx, size_t &ny,
                                size_t &nd) {
    std::memset(&op.px, 0, sizeof op.px);
    std::memset(&op.py, 0, sizeof op.py);
    std::memset(&op.post, 0, sizeof op.post);
    std::memset(&op.g, 0, sizeof op.g);
    int bpos = X.beta && Y.beta ? 1 : X.beta ? 2 : Y.beta ? 3 : 0;
    if (out_beta != (bpos != 0)) return "batch label placement";
    auto prod = [&](const Labels &l) {
        int64_t q = 1;
        for (int v : l) q *= card[v];
        return q;
    };
    const int64_t NB = nbeta;
    int64_t B = prod(bt) * (bpos == 1 ? NB : 1);
    int64_t R = prod(rows) * (bpos == 2 ? NB : 1);
    int64_t C = prod(cols) * (bpos == 3 ? NB : 1);
    int64_t K = prod(red);
    int64_t Kld = (K + 7) & ~(int64_t)7;
    int gsz = gemm_t == E_F64 ? 8 : gemm_t == E_F32 ? 4 : 2;
    int ssz = store_t == E_F64 ? 8 : 4;
    auto prep = [&](const Opnd &O, const Labels &mid, bool beta_mid, PDesc &p) -> std::string {
        std::vector<PDim> dims;
        auto push = [&](int64_t sz, int64_t sin, bool beta) { dims.push_back({sz, sin, 0, beta}); };
        if (bpos == 1) push(NB, O.per, true);
        for (int v : bt) push(card[v], stride_in(card, *O.lab, v), false);
        if (beta_mid) push(NB, O.per, true);
        for (int v : mid) push(card[v], stride_in(card, *O.lab, v), false);
        size_t nred = red.size();
        for (int v : red) push(card[v], stride_in(card, *O.lab, v), false);
        int64_t acc = 1;
        for (int i = (int)dims.size() - 1; i >= 0; --i) {
            dims[i].sout = acc;
            acc *= dims[i].sz;
            if (i == (int)(dims.size() - nred)) acc = acc / K * Kld;   // padded K row
        }
        if (nred == 0) return "GEMM without a summed label";
        std::string e = fill_pdesc(dims, p);
        if (!e.empty()) return e;
        if (!O.beta) p.beta_dim = -1;
        p.mxi = O.mx;
        p.mxi_bs = O.beta ? 1 : 0;
        p.in_type = store_t;
        p.out_type = gemm_t;
        p.in = O.ptr;
        p.out = nullptr;   // workspace, patched after allocation
        return "";
    };
    std::string e = prep(X, rows, bpos == 2, op.px);
    if (!e.empty()) return e;
    e = prep(Y, cols, bpos == 3, op.py);
    if (!e.empty()) return e;
    op.prep_bytes = (double)(B * R * K + B * C * K) * (ssz + gsz);
    GDesc &g = op.g;
    g.R = R;
    g.C = C;
    g.K = K;
    g.batch = B;
    g.ldx = g.ldy = Kld;
    g.bsx = R * Kld;
    g.bsy = C * Kld;
    g.xtype = gemm_t;
    // canonical label sequence of D ([b][r][c]); -1 marks the batch label
    std::vector<int> canon, target;
    if (bpos == 1) canon.push_back(-1);
    canon.insert(canon.end(), bt.begin(), bt.end());
    if (bpos == 2) canon.push_back(-1);
    canon.insert(canon.end(), rows.begin(), rows.end());
    if (bpos == 3) canon.push_back(-1);
    canon.insert(canon.end(), cols.begin(), cols.end());
    if (out_beta) target.push_back(-1);
    target.insert(target.end(), out_lab.begin(), out_lab.end());
    op.direct = canon == target && bpos != 3;
    g.ldd = C;
    g.bsd = R * C;
    if (op.direct) {
        g.D = out_ptr;
        g.mxd = out_mx;
        g.beta_div_batch = bpos == 1 ? B / NB : 0;
        g.beta_div_row = bpos == 2 ? R / NB : 0;
        op.has_post = false;
        nd = 0;
    } else {
        g.D = nullptr;     // workspace
        g.mxd = nullptr;
        // scatter D into the target layout
        std::vector<int64_t> cst(canon.size());
        int64_t acc = 1;
        for (int i = (int)canon.size() - 1; i >= 0; --i) {
            cst[i] = acc;
            acc *= canon[i] < 0 ? NB : card[canon[i]];
        }
        auto cstride = [&](int v) {
            for (size_t i = 0; i < canon.size(); ++i)
                if (canon[i] == v) return cst[i];
            return (int64_t)-1;
        };
        std::vector<PDim> dims;
        for (int v : target) dims.push_back({v < 0 ? NB : card[v], cstride(v), 0, v < 0});
        acc = 1;
        for (int i = (int)dims.size() - 1; i >= 0; --i) {
            dims[i].sout = acc;
            acc *= dims[i].sz;
        }
        for (auto &x : dims)
            if (x.sin < 0) return "GEMM output label missing";
        e = fill_pdesc(dims, op.post);
        if (!e.empty()) return e;
        op.post.mxi = nullptr;
        op.post.mxo = out_mx;
        op.post.in_type = store_t;
        op.post.out_type = store_t;
        op.post.in = nullptr;    // workspace
        op.post.out = out_ptr;
        op.has_post = true;
        op.post_bytes = (double)B * R * C * ssz * 2;
        nd = (size_t)(B * R * C) * ssz;
    }
    // X already laid out as [batch][rows][K] in the GEMM input type (an
    // identity preparation), 16-byte aligned, one scale for all items: the
    // GEMM reads it in place and applies the scale to D
    if (op.px.nd == 1 && op.px.sin[0] == 1 && op.px.sout[0] == 1 && K == Kld &&
        store_t == gemm_t && !X.beta && X.ptr && ((uintptr_t)X.ptr & 15) == 0) {
        op.x_in_place = true;
        op.g.X = X.ptr;
        op.g.mxsx = X.mx;
        op.prep_bytes -= (double)(B * R * K) * (ssz + gsz);
    }
    plan_permute_tiles(op.px, op.tpx);
    plan_permute_tiles(op.py, op.tpy);
    if (op.has_post) plan_permute_tiles(op.post, op.tpost);
    nx = (size_t)(B * R * Kld) * gsz;
    ny = (size_t)(B * C * Kld) * gsz;
    return "";
}

// ----------------------------------------------------- streaming kernels

struct SDim { int64_t sz, s0, s1, s2; };

static std::vector<SDim> fuse3(const std::vector<SDim> &raw) {
    std::vector<SDim> out;
    for (auto &x : raw) {
        if (x.sz == 1) continue;
        if (!out.empty()) {
            SDim &c = out.back();
            if (c.s0 == x.s0 * x.sz && c.s1 == x.s1 * x.sz && c.s2 == x.s2 * x.sz &&
                c.sz * x.sz < (1LL << 31)) {
                c.sz *= x.sz;
                c.s0 = x.s0;
                c.s1 = x.s1;
                c.s2 = x.s2;
                continue;
            }
        }
        out.push_back(x);
    }
    return out;
}

static int64_t sin_or0(const std::vector<int> &card, const Labels &l, const std::set<int> &s, int v) {
    return s.count(v) ? stride_in(card, l, v) : 0;
}

// Flat offsets of every combination of `labs` (row-major) in two tensors.
template <typename O>
static bool combo_offsets(const std::vector<int> &card, const Labels &labs, const Labels &l0,
                          const std::set<int> &s0, const Labels &l1, const std::set<int> &s1,
                          int maxn, int &n, O *o0, O *o1) {
    int64_t tot = 1;
    for (int v : labs) tot *= card[v];
    if (tot > maxn) return false;
    n = (int)tot;
    for (int64_t i = 0; i < tot; ++i) {
        int64_t r = i, a = 0, b = 0;
        for (int k = (int)labs.size() - 1; k >= 0; --k) {
            int v = labs[k];
            int64_t dg = r % card[v];
            r /= card[v];
            a += dg * sin_or0(card, l0, s0, v);
            b += dg * sin_or0(card, l1, s1, v);
        }
        if ((int64_t)(O)a != a || (int64_t)(O)b != b) return false;
        o0[i] = (O)a;
        o1[i] = (O)b;
    }
    return true;
}

// Why the last make_absorb call declined (plan trace only).
static thread_local const char *absorb_reject = "";

// Absorb: X streamed once, W small; Y's labels = R (from X) + T (new).
static bool make_absorb(const std::vector<int> &card, const Labels &lx, bool bx, int64_t perx,
                        const void *X, const unsigned long long *mxx, const Labels &lw, bool bw,
                        int64_t perw, const void *W, const unsigned long long *mxw,
                        const Labels &ly, bool by, int64_t pery, void *Y,
                        unsigned long long *mxy, const Labels *sorder, int nbeta,
                        int32_t *argmax, ADesc &d, bool dense_ok = false) {
    std::memset(&d, 0, sizeof d);
    if (by != (bx || bw)) { absorb_reject = "batch label"; return false; }
    std::set<int> sx(lx.begin(), lx.end()), sw(lw.begin(), lw.end()), sy(ly.begin(), ly.end());
    Labels R, T, S;
    for (int v : ly) (sx.count(v) ? R : T).push_back(v);
    // summed combinations in the elimination order where an argmax records a
    // flat index over them; otherwise W-only labels first, then X's summed
    // labels in X's order (X's fastest summed labels enumerate fastest, so
    // their offsets run contiguously where X stores them so)
    if (sorder && argmax) S = *sorder;
    else {
        for (int v : lw)
            if (!sy.count(v) && !sx.count(v)) S.push_back(v);
        for (int v : lx)
            if (!sy.count(v)) S.push_back(v);
    }
    if (!combo_offsets(card, S, lx, sx, lw, sw, AMAX, d.ns, d.xoff, d.wso)) { absorb_reject = "summed combinations"; return false; }
    if (!combo_offsets(card, T, ly, sy, lw, sw, AMAX, d.nt, d.yoff, d.wto)) { absorb_reject = "new combinations"; return false; }
    // more than 256 combinations: the dense kernel (sum-product, W holding
    // no position label; checked below)
    bool dense = false;
    {
        int ps = 1, pt = 1;
        while (ps < d.ns) ps <<= 1;
        while (pt < d.nt) pt <<= 1;
        dense = ps * pt > 256;
        if (dense && !dense_ok) { absorb_reject = "combination product"; return false; }
    }
    std::vector<SDim> raw;
    for (int v : R)
        raw.push_back({card[v], stride_in(card, lx, v), stride_in(card, ly, v),
                       sin_or0(card, lw, sw, v)});
    auto f = fuse3(raw);
    // inner dims: the fastest dims, at most 2048 positions (a dim that would
    // overflow that is split into (outer part, inner part)); their offset
    // table (12 bytes a position) stays under the 48 KB shared-memory default
    int ninner = 0;
    {
        int64_t nin = 1;
        int k = (int)f.size() - 1;
        while (k >= 0) {
            if (nin * f[k].sz <= 2048) {
                nin *= f[k].sz;
                ++ninner;
                --k;
                continue;
            }
            int64_t lo = 2048 / nin;
            while (lo > 1 && f[k].sz % lo) --lo;
            if (lo >= 2) {
                SDim hi{f[k].sz / lo, f[k].s0 * lo, f[k].s1 * lo, f[k].s2 * lo};
                SDim lw2{lo, f[k].s0, f[k].s1, f[k].s2};
                f[k] = hi;
                f.insert(f.begin() + k + 1, lw2);
                ++ninner;
            }
            break;
        }
    }
    if ((int)f.size() > MAXD) { absorb_reject = "too many dims"; return false; }
    d.nrd = (int)f.size();
    d.nr = 1;
    bool p2 = true;
    for (auto &x : f) {
        d.nr *= x.sz;
        p2 = p2 && (x.sz & (x.sz - 1)) == 0;
    }
    d.pow2r = p2;
    int sh = 0;
    for (int i = d.nrd - 1; i >= 0; --i) {
        d.rsz[i] = (int32_t)f[i].sz;
        d.rsx[i] = f[i].s0;
        d.rsy[i] = f[i].s1;
        d.rsw[i] = f[i].s2;
        d.rsh[i] = sh;
        if (p2) sh += __builtin_ctzll((unsigned long long)f[i].sz);
    }
    // inner offsets (shared-memory table) must fit 32 bits
    d.nin = 1;
    d.nin_d = ninner;
    int64_t ex = 0, ey = 0, ew = 0;
    for (int i = d.nrd - 1; i >= d.nrd - ninner; --i) {
        ex += (f[i].sz - 1) * f[i].s0;
        ey += (f[i].sz - 1) * f[i].s1;
        ew += (f[i].sz - 1) * f[i].s2;
        d.nin *= f[i].sz;
    }
    if (ex >= (1LL << 31) || ey >= (1LL << 31) || ew >= (1LL << 31)) { absorb_reject = "32-bit inner offsets"; return false; }
    d.nouter = d.nr / d.nin;
    // shared-label combinations (R dims that W holds), mixed radix, last fastest
    {
        int64_t c = 1;
        for (int i = d.nrd - 1; i >= 0; --i) {
            d.rshc[i] = f[i].s2 ? (int32_t)c : 0;
            if (f[i].s2) c *= f[i].sz;
            if (c >= (1LL << 30)) { absorb_reject = "shared combinations"; return false; }
        }
        d.nsh = (int)c;
    }
    if (dense && d.nsh != 1) { absorb_reject = "combination product"; return false; }
    d.nbeta = by ? nbeta : 1;
    d.bsx = (by && bx) ? perx : 0;
    d.bsw = (by && bw) ? perw : 0;
    d.bsy = by ? pery : 0;
    d.X = X;
    d.W = W;
    d.Y = Y;
    d.mxx = mxx;
    d.mxw = mxw;
    d.mxx_bs = bx ? 1 : 0;
    d.mxw_bs = bw ? 1 : 0;
    d.mxy = mxy;
    d.argmax = argmax;
    return true;
}

// Reduce: O[g, s, t] = sum_m X[g, m, s] Z[g, m, t].
static bool make_reduce(const std::vector<int> &card, const Labels &lx, bool bx, int64_t perx,
                        const void *X, const unsigned long long *mxx, const Labels &lz, bool bz,
                        int64_t perz, const void *Z, const unsigned long long *mxz,
                        const Labels &lo, bool bo, int64_t pero, void *O,
                        unsigned long long *mxo, int nbeta, RDesc &d) {
    std::memset(&d, 0, sizeof d);
    if (bo != (bx || bz)) return false;
    std::set<int> sx(lx.begin(), lx.end()), sz(lz.begin(), lz.end()), so(lo.begin(), lo.end());
    Labels G, S, T, M;
    for (int v : lo) {
        bool ix = sx.count(v), iz = sz.count(v);
        if (ix && iz) G.push_back(v);
        else if (ix) S.push_back(v);
        else if (iz) T.push_back(v);
        else return false;
    }
    for (int v : lx)
        if (!so.count(v)) M.push_back(v);
    for (int v : lz)
        if (!so.count(v) && !sx.count(v)) M.push_back(v);
    if (!combo_offsets(card, S, lx, sx, lo, so, AMAX, d.ns, d.xoff, d.oso)) return false;
    if (!combo_offsets(card, T, lz, sz, lo, so, AMAX, d.nt, d.zoff, d.oto)) return false;
    std::vector<SDim> g, m;
    for (int v : G) g.push_back({card[v], stride_in(card, lx, v), stride_in(card, lz, v), stride_in(card, lo, v)});
    for (int v : M) m.push_back({card[v], sin_or0(card, lx, sx, v), sin_or0(card, lz, sz, v), 0});
    auto fg = fuse3(g), fm = fuse3(m);
    // inner summed dims (offset table of at most 2048 positions)
    int ninner = 0;
    {
        int64_t nin = 1;
        int k = (int)fm.size() - 1;
        while (k >= 0) {
            if (nin * fm[k].sz <= 2048) {
                nin *= fm[k].sz;
                ++ninner;
                --k;
                continue;
            }
            int64_t lo = 2048 / nin;
            while (lo > 1 && fm[k].sz % lo) --lo;
            if (lo >= 2) {
                SDim hi{fm[k].sz / lo, fm[k].s0 * lo, fm[k].s1 * lo, 0};
                SDim lw2{lo, fm[k].s0, fm[k].s1, 0};
                fm[k] = hi;
                fm.insert(fm.begin() + k + 1, lw2);
                ++ninner;
            }
            break;
        }
    }
    if ((int)fg.size() > MAXD || (int)fm.size() > MAXD) return false;
    d.ngd = (int)fg.size();
    d.ng = 1;
    for (int i = 0; i < d.ngd; ++i) {
        d.gsz[i] = (int32_t)fg[i].sz;
        d.gsx[i] = fg[i].s0;
        d.gsz2[i] = fg[i].s1;
        d.gso[i] = fg[i].s2;
        d.ng *= fg[i].sz;
    }
    d.nmd = (int)fm.size();
    d.nm = 1;
    bool p2 = true;
    for (auto &x : fm) {
        d.nm *= x.sz;
        p2 = p2 && (x.sz & (x.sz - 1)) == 0;
    }
    d.pow2m = p2;
    int sh = 0;
    for (int i = d.nmd - 1; i >= 0; --i) {
        d.msz[i] = (int32_t)fm[i].sz;
        d.msx[i] = fm[i].s0;
        d.msz2[i] = fm[i].s1;
        d.msh[i] = sh;
        if (p2) sh += __builtin_ctzll((unsigned long long)fm[i].sz);
    }
    d.nin_d = ninner;
    d.nin = 1;
    int64_t ex = 0, ez = 0;
    for (int i = d.nmd - 1; i >= d.nmd - ninner; --i) {
        ex += (fm[i].sz - 1) * fm[i].s0;
        ez += (fm[i].sz - 1) * fm[i].s1;
        d.nin *= fm[i].sz;
    }
    if (ex >= (1LL << 31) || ez >= (1LL << 31)) return false;
    d.nouter = d.nm / d.nin;
    d.nbeta = bo ? nbeta : 1;
    d.bsx = (bo && bx) ? perx : 0;
    d.bsz = (bo && bz) ? perz : 0;
    d.bso = bo ? pero : 0;
    d.X = X;
    d.Z = Z;
    d.O = O;
    d.mxx = mxx;
    d.mxz = mxz;
    d.mxx_bs = bx ? 1 : 0;
    d.mxz_bs = bz ? 1 : 0;
    d.mxo = mxo;
    return true;
}

// Batched strided GEMM: O[g, m, n] = sum_k X[g, m, k] Y[g, k, n] with the
// label groups G (in X, Y and O), M (X and O), N (Y and O) and K (X and Y),
// each label of O, X and Y in exactly one group (no label summed inside one
// operand).  The side with more row entries goes to M.  Writes the offset
// tables, in the order the descriptor's table pointers take them, to `tab`.
static bool make_bgemm(const std::vector<int> &card, const Labels &lx, bool bx, int64_t perx,
                       const void *X, const unsigned long long *mxx, const Labels &ly, bool by,
                       int64_t pery, const void *Y, const unsigned long long *mxy,
                       const Labels &lo, bool bo, int64_t pero, void *O,
                       unsigned long long *mxo, int nbeta, int esz, BDesc &d,
                       std::vector<int32_t> &tab, bool tc_orient = false,
                       bool swapped = false) {
    std::memset(&d, 0, sizeof d);
    if (bo != (bx || by)) return false;
    std::set<int> sx(lx.begin(), lx.end()), sy(ly.begin(), ly.end()), so(lo.begin(), lo.end());
    Labels G, M, N, K;
    for (int v : lx) {
        bool iy = sy.count(v), io = so.count(v);
        if (iy && io) G.push_back(v);
        else if (io) M.push_back(v);
        else if (iy) K.push_back(v);
        else return false;
    }
    for (int v : ly) {
        bool ix = sx.count(v), io = so.count(v);
        if (ix) continue;
        if (io) N.push_back(v);
        else return false;
    }
    for (int v : lo)
        if (!sx.count(v) && !sy.count(v)) return false;
    auto prod = [&](const Labels &l) {
        int64_t p = 1;
        for (int v : l) p *= card[v];
        return p;
    };
    d.G = prod(G);
    d.M = prod(M);
    d.N = prod(N);
    d.K = prod(K);
    // orientation: for the tensor-core gather kernel (float data, epilogue
    // storing along M) the output's fastest label on the M side; for the
    // CUDA-core kernel the larger side on M
    auto fastest_of = [&](const Labels &lt) {
        for (int k = (int)lt.size() - 1; k >= 0; --k)
            if (card[lt[k]] > 1) return lt[k];
        return -1;
    };
    const int fo = fastest_of(lo);
    const bool o_in_n = std::find(N.begin(), N.end(), fo) != N.end();
    const bool o_in_m = std::find(M.begin(), M.end(), fo) != M.end();
    if (!swapped && (tc_orient && esz == 4 ? (o_in_n || (!o_in_m && d.N > d.M)) : d.N > d.M))
        return make_bgemm(card, ly, by, pery, Y, mxy, lx, bx, perx, X, mxx, lo, bo, pero, O, mxo,
                          nbeta, esz, d, tab, tc_orient, true);
    if (perx >= (1LL << 31) || pery >= (1LL << 31) || pero >= (1LL << 31)) return false;
    const int64_t ntab = 3 * d.G + 2 * d.M + 2 * d.N + 2 * d.K;
    if (ntab > (1LL << 26)) return false;
    tab.assign((size_t)ntab, 0);
    // offsets of every index of a group (labels in the given order, last
    // fastest) in one tensor
    auto fill = [&](const Labels &grp, const Labels &lt, const std::set<int> &st, int32_t *out) {
        int64_t tot = prod(grp);
        std::vector<int64_t> sz, sd;
        for (int v : grp) {
            sz.push_back(card[v]);
            sd.push_back(st.count(v) ? stride_in(card, lt, v) : 0);
        }
        std::vector<int64_t> dig(grp.size(), 0);
        int64_t off = 0;
        for (int64_t i = 0; i < tot; ++i) {
            out[i] = (int32_t)off;
            for (int k = (int)grp.size() - 1; k >= 0; --k) {
                off += sd[k];
                if (++dig[k] < sz[k]) break;
                off -= sd[k] * sz[k];
                dig[k] = 0;
            }
        }
    };
    int32_t *t = tab.data();
    int64_t p = 0;
    int64_t o_ag = p; fill(G, lx, sx, t + p); p += d.G;
    int64_t o_bg = p; fill(G, ly, sy, t + p); p += d.G;
    int64_t o_cg = p; fill(G, lo, so, t + p); p += d.G;
    int64_t o_am = p; fill(M, lx, sx, t + p); p += d.M;
    int64_t o_cm = p; fill(M, lo, so, t + p); p += d.M;
    int64_t o_bn = p; fill(N, ly, sy, t + p); p += d.N;
    int64_t o_cn = p; fill(N, lo, so, t + p); p += d.N;
    int64_t o_ak = p; fill(K, lx, sx, t + p); p += d.K;
    int64_t o_bk = p; fill(K, ly, sy, t + p); p += d.K;
    // table pointers hold offsets into the table until the buffer is placed
    d.tag = (const int32_t *)(intptr_t)o_ag;
    d.tbg = (const int32_t *)(intptr_t)o_bg;
    d.tcg = (const int32_t *)(intptr_t)o_cg;
    d.tam = (const int32_t *)(intptr_t)o_am;
    d.tcm = (const int32_t *)(intptr_t)o_cm;
    d.tbn = (const int32_t *)(intptr_t)o_bn;
    d.tcn = (const int32_t *)(intptr_t)o_cn;
    d.tak = (const int32_t *)(intptr_t)o_ak;
    d.tbk = (const int32_t *)(intptr_t)o_bk;
    // the group holding each tensor's fastest label (of size > 1)
    auto fastest = [&](const Labels &lt) {
        for (int k = (int)lt.size() - 1; k >= 0; --k)
            if (card[lt[k]] > 1) return lt[k];
        return -1;
    };
    auto in = [](const Labels &l, int v) { return std::find(l.begin(), l.end(), v) != l.end(); };
    d.a_kfast = in(K, fastest(lx)) ? 1 : 0;
    d.b_kfast = in(K, fastest(ly)) ? 1 : 0;
    d.c_nfast = in(N, fastest(lo)) ? 1 : 0;
    // a group label inside C's 32-byte sectors: tiles enumerate G fastest,
    // so the tiles sharing a sector write it at about the same time
    d.c_gfast = 0;
    for (int v : G)
        if (card[v] > 1 && stride_in(card, lo, v) * esz < 32) d.c_gfast = 1;
    d.nbeta = bo ? nbeta : 1;
    d.bsa = (bo && bx) ? perx : 0;
    d.bsb = (bo && by) ? pery : 0;
    d.bsc = bo ? pero : 0;
    d.A = X;
    d.B = Y;
    d.C = O;
    d.mxa = mxx;
    d.mxb = mxy;
    d.mxa_bs = bx ? 1 : 0;
    d.mxb_bs = by ? 1 : 0;
    d.mxc = mxo;
    bgemm_configure(d, esz);
    return d.tile >= 0;
}

static bool to_micro(const CDesc &d, const char *arena, int esz, const unsigned long long *mxb,
                     const int32_t *amb, MicroDesc &m) {
    std::memset(&m, 0, sizeof m);
    if (d.nout > MICRO_D || d.nk > MICRO_D || d.nbeta > MICRO_BETA) return false;
    if (d.nout_total * d.nbeta > MICRO_MAX || d.ktotal > (1LL << 30)) return false;
    m.nout = d.nout;
    m.nk = d.nk;
    m.pow2 = d.pow2;
    m.nbeta = d.nbeta;
    m.nout_total = (int32_t)d.nout_total;
    m.ktotal = (int32_t)d.ktotal;
    m.offA = ((const char *)d.A - arena) / esz;
    m.offB = ((const char *)d.B - arena) / esz;
    m.offC = ((const char *)d.C - arena) / esz;
    m.bsa = (int32_t)d.bsa;
    m.bsb = (int32_t)d.bsb;
    for (int i = 0; i < d.nout; ++i) {
        m.osz[i] = d.osz[i];
        m.osh[i] = d.osh[i];
        m.osa[i] = (int32_t)d.osa[i];
        m.osb[i] = (int32_t)d.osb[i];
    }
    for (int i = 0; i < d.nk; ++i) {
        m.ksz[i] = d.ksz[i];
        m.ksh[i] = d.ksh[i];
        m.ksa[i] = (int32_t)d.ksa[i];
        m.ksb[i] = (int32_t)d.ksb[i];
    }
    m.mxa = d.mxa ? d.mxa - mxb : -1;
    m.mxb = d.mxb ? d.mxb - mxb : -1;
    m.mxc = d.mxc ? d.mxc - mxb : -1;
    m.mxa_bs = d.mxa_bs;
    m.mxb_bs = d.mxb_bs;
    m.amoff = d.argmax ? d.argmax - amb : -1;
    return true;
}

// Inner offset tables of the streaming kernels (computed once per node).
// Chunk table of one operand tile of a dense kernel (dense_impl.cuh): tiles
// are P consecutive inner positions; entry (p, v) of a tile sits at
// pos[c P + p] + voff[v] from the operand's base, which must be the tile's
// base pos[c P] (a multiple of 4) plus a pattern that is the same for every
// tile c.  Sorted by offset, the pattern's entries must form whole, aligned
// quads of consecutive entries.  Appends the quads' offsets [nq] and, per
// quad, the shared-memory slots (row0 + v) * RS + p of its four entries
// (16-bit, [nq][4]) to `out` (even-aligned) and returns the table position,
// or -1 when the pattern does not chunk.
template <typename O>
static int dense_chunks(const std::vector<int64_t> &pos, int P, const O *voff, int nv, int RS,
                        int row0, bool base4, std::vector<int32_t> &out) {
    const int64_t nin = (int64_t)pos.size();
    if (!base4 || nin % P || nv < 1) return -1;
    for (int64_t c = 0; c < nin; c += P) {
        if (pos[c] % 4) return -1;
        for (int p = 0; p < P; ++p)
            if (pos[c + p] - pos[c] != pos[p] - pos[0]) return -1;
    }
    struct E { int64_t off; int slot; };
    std::vector<E> es;
    es.reserve((size_t)P * nv);
    for (int v = 0; v < nv; ++v) {
        for (int p = 0; p < P; ++p)
            es.push_back({pos[p] - pos[0] + (int64_t)voff[v], (row0 + v) * RS + p});
    }
    std::sort(es.begin(), es.end(), [](const E &a, const E &b) { return a.off < b.off; });
    if (es.size() % 4) return -1;
    const size_t nq = es.size() / 4;
    for (size_t q = 0; q < nq; ++q) {
        const int64_t o = es[4 * q].off;
        if (o % 4 || o >= (1LL << 31)) return -1;
        for (int i = 1; i < 4; ++i)
            if (es[4 * q + i].off != o + i) return -1;
    }
    if (out.size() % 2) out.push_back(0);
    const int at = (int)out.size();
    out.resize(out.size() + 3 * nq, 0);
    uint16_t *sl = (uint16_t *)(out.data() + at + nq);
    for (size_t q = 0; q < nq; ++q) {
        out[at + q] = (int32_t)es[4 * q].off;
        for (int i = 0; i < 4; ++i) sl[4 * q + i] = (uint16_t)es[4 * q + i].slot;
    }
    return at;
}

static void absorb_table(ADesc &d, int esz, std::vector<int32_t> &out) {
    const int nin = (int)d.nin, nod = d.nrd - d.nin_d;
    out.assign((size_t)4 * nin + d.nsh, 0);
    for (int i = 0; i < nin; ++i) {
        int64_t r = i, x0 = 0, y0 = 0, w0 = 0, c0 = 0;
        for (int k = d.nrd - 1; k >= nod; --k) {
            int64_t dg = r % d.rsz[k];
            r /= d.rsz[k];
            x0 += dg * d.rsx[k];
            y0 += dg * d.rsy[k];
            w0 += dg * d.rsw[k];
            c0 += dg * d.rshc[k];
        }
        out[i] = (int32_t)x0;
        out[nin + i] = (int32_t)y0;
        out[2 * nin + i] = (int32_t)w0;
        out[3 * nin + i] = (int32_t)c0;
    }
    // W offset of each shared-label combination
    for (int c = 0; c < d.nsh; ++c) {
        int64_t r = c, w0 = 0;
        for (int k = d.nrd - 1; k >= 0; --k) {
            if (!d.rshc[k]) continue;
            int64_t dg = r % d.rsz[k];
            r /= d.rsz[k];
            w0 += dg * d.rsw[k];
        }
        out[4 * nin + c] = (int32_t)w0;
    }
    // chunked tile copies of the dense absorb
    d.cx = d.cy = 0;
    if (absorb_dense_form_host(d)) {
        const int P = 128, RS = P + 16 / esz;
        const int nod2 = d.nrd - d.nin_d;
        auto base4 = [&](const int64_t *st, int64_t bs, const void *ptr) {
            if (bs % 4 || ((uintptr_t)ptr & 15)) return false;
            for (int k = 0; k < nod2; ++k)
                if (st[k] % 4) return false;
            return true;
        };
        std::vector<int64_t> px(out.begin(), out.begin() + nin),
            py(out.begin() + nin, out.begin() + 2 * nin);
        int at = dense_chunks(px, P, d.xoff, d.ns, RS, 0, base4(d.rsx, d.bsx, d.X), out);
        if (at >= 0) {
            d.cx = 1;
            d.cxo = at;
        }
        at = dense_chunks(py, P, d.yoff, d.nt, RS, 0, base4(d.rsy, d.bsy, d.Y), out);
        if (at >= 0) {
            d.cy = 1;
            d.cyo = at;
        }
    }
}

static void reduce_table(RDesc &d, int esz, std::vector<int32_t> &out) {
    const int nin = (int)d.nin, nod = d.nmd - d.nin_d;
    out.assign((size_t)2 * nin, 0);
    for (int i = 0; i < nin; ++i) {
        int64_t r = i, x0 = 0, z0 = 0;
        for (int k = d.nmd - 1; k >= nod; --k) {
            int64_t dg = r % d.msz[k];
            r /= d.msz[k];
            x0 += dg * d.msx[k];
            z0 += dg * d.msz2[k];
        }
        out[i] = (int32_t)x0;
        out[nin + i] = (int32_t)z0;
    }
    // chunked tile copies of the dense reduce
    d.cx = d.cz = 0;
    if (reduce_dense_describe(d) >= 0) {
        const int P = 64, RR = P + 16 / esz;
        auto base4 = [&](const int64_t *ms, const int64_t *gs, int64_t bs, const void *ptr) {
            if (bs % 4 || ((uintptr_t)ptr & 15)) return false;
            for (int k = 0; k < nod; ++k)
                if (ms[k] % 4) return false;
            for (int k = 0; k < d.ngd; ++k)
                if (gs[k] % 4) return false;
            return true;
        };
        std::vector<int64_t> px(out.begin(), out.begin() + nin),
            pz(out.begin() + nin, out.begin() + 2 * nin);
        int at = dense_chunks(px, P, d.xoff, d.ns, RR, 0, base4(d.msx, d.gsx, d.bsx, d.X), out);
        if (at >= 0) {
            d.cx = 1;
            d.cxo = at;
        }
        at = dense_chunks(pz, P, d.zoff, d.nt, RR, 32, base4(d.msz2, d.gsz2, d.bsz, d.Z), out);
        if (at >= 0) {
            d.cz = 1;
            d.czo = at;
        }
    }
}

// TN_PLAN_TRACE=1 prints every step of a built program to stderr (one line
// per step: direction, kernel family, shape parameters, algorithmic cost).
static void trace_program(const Program &P) {
    const char *e = getenv("TN_PLAN_TRACE");
    if (!e || e[0] != '1') return;
    int i = 0;
    for (auto *steps : {&P.fsteps, &P.bsteps}) {
        const char *dir = steps == &P.fsteps ? "fwd" : "bwd";
        for (auto &st : *steps) {
            if (st.kind == 2) {
                const ADesc &a = st.ad;
                fprintf(stderr, "%s %d absorb ns %d nt %d nr %lld nin %lld nouter %lld beta %d nsh %d",
                        dir, i, a.ns, a.nt, (long long)a.nr, (long long)a.nin,
                        (long long)a.nouter, a.nbeta, a.nsh);
                fprintf(stderr, " xoff");
                for (int k = 0; k < a.ns && k < 8; ++k) fprintf(stderr, ",%d", a.xoff[k]);
                fprintf(stderr, " yoff");
                for (int k = 0; k < a.nt && k < 8; ++k) fprintf(stderr, ",%d", a.yoff[k]);
                {
                    int xm, ym;
                    absorb_dense_describe(a, xm, ym);
                    if (xm >= 0) fprintf(stderr, " dense x%d y%d", xm, ym);
                }
                fprintf(stderr, " rdims");
                for (int k = 0; k < a.nrd; ++k)
                    fprintf(stderr, ",%d:%lld/%lld/%lld", a.rsz[k], (long long)a.rsx[k],
                            (long long)a.rsy[k], (long long)a.rsw[k]);
            } else if (st.kind == 3) {
                const RDesc &r = st.rd;
                fprintf(stderr, "%s %d reduce ns %d nt %d ng %lld nm %lld nin %lld beta %d vec %d",
                        dir, i, r.ns, r.nt, (long long)r.ng, (long long)r.nm, (long long)r.nin,
                        r.nbeta, (int)reduce_vector_form(r, P.esz));
                fprintf(stderr, " xoff");
                for (int k = 0; k < r.ns && k < 8; ++k) fprintf(stderr, ",%lld", (long long)r.xoff[k]);
                fprintf(stderr, " zoff");
                for (int k = 0; k < r.nt && k < 8; ++k) fprintf(stderr, ",%lld", (long long)r.zoff[k]);
                if (reduce_dense_describe(r) >= 0) fprintf(stderr, " dense v%d", reduce_dense_describe(r));
                fprintf(stderr, " mdims");
                for (int k = 0; k < r.nmd; ++k)
                    fprintf(stderr, ",%d:%lld/%lld", r.msz[k], (long long)r.msx[k],
                            (long long)r.msz2[k]);
            }
            else if (st.kind == 1) {
                fprintf(stderr, "%s %d gemm%s b %lld m %lld n %lld k %lld", dir, i,
                        st.g.tc ? "-tc" : "-simt", (long long)st.g.g.batch, (long long)st.g.g.R,
                        (long long)st.g.g.C, (long long)st.g.g.K);
                auto pd = [](const char *nm, const PDesc &q) {
                    fprintf(stderr, " | %s%s", nm, q.tl.tn > 0 ? "(tiled)" : "");
                    for (int k = 0; k < q.nd; ++k)
                        fprintf(stderr, " %d:%lld>%lld", q.sz[k], (long long)q.sin[k],
                                (long long)q.sout[k]);
                };
                pd("px", st.g.px);
                pd("py", st.g.py);
                if (st.g.has_post) pd("post", st.g.post);
            }
            else if (st.kind == 4) {
                const BDesc &b = st.bd;
                fprintf(stderr, "%s %d bgemm g %lld m %lld n %lld k %lld beta %d split %d tile %d "
                        "kfast %d/%d nfast %d", dir, i, (long long)b.G, (long long)b.M,
                        (long long)b.N, (long long)b.K, b.nbeta, b.nsplit, b.tile, b.a_kfast,
                        b.b_kfast, b.c_nfast);
            }
            else
                fprintf(stderr, "%s %d contract outs %lld k %lld [%s]", dir, i,
                        (long long)st.d.nout_total, (long long)st.d.ktotal, st.why);
            fprintf(stderr, " MB %.3f MFLOP %.3f lane %d waits %d\n", st.bytes / 1e6, st.flops / 1e6,
                    st.lane, (int)st.waits.size());
            ++i;
        }
    }
}

// Build (plan, allocate, describe, capture) a program.
tn_status build_program(tn_model *m, const Net &net, const Tree &tree, int kind, int dtype,
                        int nbeta, bool grads, const tn_options *opts, Program &P,
                        const std::vector<LeafRec> *spec = nullptr,
                        const Tune *tune = nullptr) {
    if (tune) P.tune = *tune;
    P.kind = kind;
    P.dtype = dtype;
    P.esz = (int)elem_bytes(dtype);
    P.nbeta = nbeta;
    P.grads = grads;
    const bool maxplus = kind == K_MAP || kind == K_MAXNET;
    tn_prec prec = opts ? opts->prec : TN_FP64;
    P.gemm_type = prec == TN_FP64 ? E_F64 : prec == TN_BF16 ? E_BF16 : E_F32;
    const bool use_tc = prec == TN_TF32 || prec == TN_BF16;
    std::string err = build_plan(net, tree, P.plan, maxplus ? 0 : 64);
    if (!err.empty()) return fail(TN_E_ORDER, err);
    const Plan &pl = P.plan;
    const int n = tree.nleaves;
    const int NN = 2 * n - 1;
    const bool backward = kind == K_MAR;
    const bool keep_all = kind != K_PR && kind != K_SUMNET;
    P.fwd.assign(NN, Slot());
    P.adj.assign(NN, Slot());
    // ---- maxima slots
    int64_t nmx = 0;
    for (int id = 0; id < NN; ++id) {
        Slot &s = P.fwd[id];
        s.per = pl.node[id].size;
        s.beta = pl.node[id].beta;
        s.elems = s.per * (s.beta ? nbeta : 1);
        s.mx = nmx;
        nmx += s.beta ? nbeta : 1;
    }
    // adjoint batch flags and which adjoints are needed
    P.adj_beta.assign(NN, 0);
    P.need_adj.assign(NN, 0);
    if (backward) {
        P.adj_beta[pl.root] = pl.node[pl.root].beta;
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            P.adj_beta[nd.a] = P.adj_beta[id] || pl.node[nd.b].beta;
            P.adj_beta[nd.b] = P.adj_beta[id] || pl.node[nd.a].beta;
        }
        for (int id = 0; id < NN; ++id) {
            bool leaf = id < n;
            bool unity = leaf && id >= (int)m->md.nfactors && kind == K_MAR;
            P.need_adj[id] = !leaf || unity || (leaf && grads && id < m->md.nfactors);
        }
        for (int id = 0; id < NN; ++id) {
            Slot &s = P.adj[id];
            s.per = pl.node[id].size;
            s.beta = P.adj_beta[id];
            s.elems = s.per * (s.beta ? nbeta : 1);
            s.mx = nmx;
            nmx += s.beta ? nbeta : 1;
        }
    }
    P.nmx = nmx;
    // ---- micro subtrees: maximal subtrees of at most MICRO_NODES nodes whose
    // tensors (and adjoints) all hold at most MICRO_MAX entries
    P.micro.assign(NN, 0);
    std::vector<int> micro_root(NN, -1);
    if (nbeta <= MICRO_BETA) {
        std::vector<char> small(NN, 0);
        std::vector<int> cnt(NN, 0);
        const int INF = 1 << 29;
        auto emax = [&](int id) {
            int64_t e = P.fwd[id].elems;
            if (backward) e = std::max(e, P.adj[id].elems);
            return e;
        };
        for (int id = n; id < NN; ++id) {
            const Node &nd = pl.node[id];
            bool ok = !nd.gemm && emax(id) <= MICRO_MAX && emax(nd.a) <= MICRO_MAX &&
                      emax(nd.b) <= MICRO_MAX && (nd.a < n || small[nd.a]) &&
                      (nd.b < n || small[nd.b]);
            small[id] = ok;
            cnt[id] = ok ? 1 + (nd.a < n ? 0 : cnt[nd.a]) + (nd.b < n ? 0 : cnt[nd.b]) : INF;
        }
        for (int id = NN - 1; id >= n; --id) {
            int par = pl.node[id].parent;
            if (par >= 0 && micro_root[par] >= 0) {
                micro_root[id] = micro_root[par];
            } else if (small[id] && cnt[id] <= MICRO_NODES) {
                micro_root[id] = id;
            }
            if (micro_root[id] >= 0) P.micro[id] = 1;
        }
    }
    std::map<int, std::vector<int>> msub;   // micro root -> its nodes (ascending)
    for (int id = n; id < NN; ++id)
        if (P.micro[id]) msub[micro_root[id]].push_back(id);
    // ---- arena offsets, in execution order: leaves, micro subtrees, the
    // other nodes in id order; adjoints in the backward's order
    std::vector<int> fwd_order, bwd_order;
    for (auto &kv : msub)
        for (int id : kv.second) fwd_order.push_back(id);
    for (int id = n; id < NN; ++id)
        if (!P.micro[id]) fwd_order.push_back(id);
    for (int id = NN - 1; id >= n; --id)
        if (!P.micro[id]) bwd_order.push_back(id);
    for (auto &kv : msub)
        for (auto it = kv.second.rbegin(); it != kv.second.rend(); ++it) bwd_order.push_back(*it);
    // ---- lanes: in PR and MAR programs the lighter child subtree of a node,
    // when it carries at least 3% of the tree's tensor entries, runs on
    // another stream of the captured graph (its steps wait for the results
    // they read through events), so independent parts of the tree overlap.
    // Memory is then never recycled, as concurrent parts would race on it.
    const int kLanes = std::max(1, std::min(4, P.tune.max_lanes));
    P.lane.assign(NN, 0);
    int nl_used = 1;
    if ((kind == K_PR || kind == K_MAR) && kLanes > 1) {
        std::vector<double> work(NN, 0.0);
        for (int id = n; id < NN; ++id) {
            const Node &nd = pl.node[id];
            work[id] = (P.micro[id] ? 0.0 : (double)P.fwd[id].elems) + work[nd.a] + work[nd.b];
        }
        const double total = work[pl.root];
        int next = 0;
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            int heavy = work[nd.a] >= work[nd.b] ? nd.a : nd.b;
            int light = heavy == nd.a ? nd.b : nd.a;
            P.lane[heavy] = P.lane[id];
            P.lane[light] = P.lane[id];
            if (light >= n && !P.micro[light] && work[light] >= 0.03 * total) {
                P.lane[light] = (P.lane[id] + 1 + (next++ % (kLanes - 1))) % kLanes;
                nl_used = kLanes;
            }
        }
    }
    P.drop.assign(NN, 0);
    P.rec_off.assign(NN, -1);
    // is fwd[c] read by the adjoint steps of its parent?  (fwd[a] by the
    // sibling's adjoint B-bar, fwd[b] by A-bar)
    auto fwd_read_back = [&](int c) {
        const int par = pl.node[c].parent;
        if (par < 0 || !backward) return false;
        const Node &pn = pl.node[par];
        return P.need_adj[c == pn.a ? pn.b : pn.a] != 0;
    };
    auto plan_arena = [&](bool recycle) {
        OffsetAlloc A;
        for (int id = 0; id < n; ++id) P.fwd[id].off = A.alloc(P.fwd[id].elems);
        // Micro subtrees run concurrently (one CTA each), so memory is never
        // recycled inside the micro phase; their tensors are tiny.
        for (int id : fwd_order) {
            const Node &nd = pl.node[id];
            P.fwd[id].off = A.alloc(P.fwd[id].elems);
            if (recycle && !keep_all && !P.micro[id]) {
                A.release(P.fwd[nd.a].off, P.fwd[nd.a].elems);
                A.release(P.fwd[nd.b].off, P.fwd[nd.b].elems);
            } else if (!P.micro[id]) {
                for (int c : {nd.a, nd.b})
                    if (P.drop[c]) A.release(P.fwd[c].off, P.fwd[c].elems);
            }
        }
        if (backward) {
            P.adj[pl.root].off = A.alloc(P.adj[pl.root].elems);
            for (int id : bwd_order) {
                const Node &nd = pl.node[id];
                for (int c : {nd.a, nd.b}) {
                    P.rec_off[c] = -1;
                    if (P.drop[c] && fwd_read_back(c)) P.rec_off[c] = A.alloc(P.fwd[c].elems);
                }
                for (int c : {nd.a, nd.b})
                    if (P.need_adj[c]) P.adj[c].off = A.alloc(P.adj[c].elems);
                if (recycle && !P.micro[id]) A.release(P.adj[id].off, P.adj[id].elems);
                for (int c : {nd.a, nd.b})
                    if (P.rec_off[c] >= 0) A.release(P.rec_off[c], P.fwd[c].elems);
            }
        }
        return A.top;
    };
    if (nl_used > 1) {
        // lanes only where the unrecycled arena stays modest
        int64_t rec = plan_arena(true), all = plan_arena(false);
        if ((double)all * P.esz > std::max(4.0e9, 1.5 * (double)rec * P.esz)) {
            nl_used = 1;
            std::fill(P.lane.begin(), P.lane.end(), 0);
        }
    }
    P.nlanes = nl_used;
    int64_t arena_top = plan_arena(nl_used == 1);
    P.keep_all_elems = arena_top;
    int64_t budget = opts ? opts->hbm_budget_bytes : 0;
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
    // the memory the program may take: the budget, else what is free
    const double limit = budget > 0 ? (double)budget : (double)freeb - (double)(256u << 20);
    auto need_of = [&](int64_t top) { return (double)top * P.esz + (double)nmx * 8; };
    if (kind == K_MAR && nbeta == 1 && need_of(arena_top) > limit) {
        // checkpointing (a batch of evidence sets is split into smaller
        // batches first, which costs no extra work): drop the largest forward
        // tensors, no two of them parent and child (a recompute reads only
        // kept tensors), until the arena fits; one lane (the arena is
        // recycled in step order)
        nl_used = 1;
        P.nlanes = 1;
        std::fill(P.lane.begin(), P.lane.end(), 0);
        arena_top = plan_arena(true);
        std::vector<int> cand;
        for (int id = n; id < NN; ++id)
            if (id != pl.root && !P.micro[id] && fwd_read_back(id)) cand.push_back(id);
        std::stable_sort(cand.begin(), cand.end(),
                         [&](int x, int y) { return P.fwd[x].elems > P.fwd[y].elems; });
        for (int c : cand) {
            if (need_of(arena_top) <= limit) break;
            const Node &cn = pl.node[c];
            if (P.drop[cn.a] || P.drop[cn.b] || (cn.parent >= 0 && P.drop[cn.parent])) continue;
            P.drop[c] = 1;
            int64_t t = plan_arena(true);
            if (t < arena_top) {
                arena_top = t;
                ++P.ndrop;
            } else {
                P.drop[c] = 0;
            }
        }
        arena_top = plan_arena(true);
    }
    P.arena_elems = arena_top;
    // argmax buffers
    int64_t am_total = 0;
    P.am_off.assign(NN, -1);
    if (maxplus)
        for (int id = n; id < NN; ++id) {
            P.am_off[id] = am_total;
            am_total += (P.fwd[id].elems + 63) & ~(int64_t)63;
        }
    // ---- budget and allocation
    size_t need = (size_t)P.arena_elems * P.esz + (size_t)nmx * 8 + (size_t)am_total * 4;
    if ((budget > 0 && (int64_t)need > budget) || need + (256u << 20) > freeb) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "program needs %.3f GB of device memory (budget %.3f GB, free %.3f GB)",
                 need / 1e9, budget / 1e9, freeb / 1e9);
        return fail(TN_E_OOM, buf);
    }
    CK(P.mem.alloc(&P.arena, (size_t)P.arena_elems * P.esz));
    CK(P.mem.alloc(&P.mx, (size_t)nmx * 8));
    if (am_total) CK(P.mem.alloc(&P.am, (size_t)am_total * 4));
    CK(P.mem.alloc(&P.d_evid, (size_t)nbeta * std::max(1, m->md.nvars) * 4));
    CK(P.mem.alloc(&P.d_slice_val, 4 * std::max<size_t>(1, m->slice_vars.size())));
    CK(cudaMemset(P.d_slice_val, 0, 4 * std::max<size_t>(1, m->slice_vars.size())));
    CK(P.mem.alloc(&P.d_logz, (size_t)nbeta * 8));
    CK(P.mem.alloc(&P.d_sigma, (size_t)nbeta * 8));
    CK(P.mem.alloc(&P.d_card, net.card.size() * 4 + 4));
    CK(cudaMemcpy(P.d_card, net.card.data(), net.card.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(P.d_evid, 0xff, (size_t)nbeta * std::max(1, m->md.nvars) * 4));
    // ---- leaf records
    for (int id = 0; id < n; ++id) {
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        r.nkd = -1;
        r.slice_of_var = -1;
        if (spec) {
            r = (*spec)[id];
            r.nkd = -1;
            r.slice_of_var = -1;
            if (r.kind == LEAF_UNITY) r.beta = pl.node[id].beta;
        } else if (id < (int)m->md.nfactors) {
            r.kind = LEAF_FACTOR;
            r.src = m->md.toff[id];
            const Labels &full = m->md.scope[id];
            if (full.size() != net.leaf[id].size()) {
                // sliced factor: gather the kept labels at the slice values
                if (full.size() > (size_t)LEAF_D)
                    return fail(TN_E_UNSUPPORTED, "sliced factor with more than 16 variables");
                r.nkd = 0;
                r.nsd = 0;
                for (int v : full) {
                    int64_t st = stride_in(m->md.card, full, v);
                    auto it = std::find(m->slice_vars.begin(), m->slice_vars.end(), v);
                    if (it != m->slice_vars.end()) {
                        r.sidx[r.nsd] = (int32_t)(it - m->slice_vars.begin());
                        r.sst[r.nsd++] = st;
                    } else {
                        r.ksz[r.nkd] = m->md.card[v];
                        r.kst[r.nkd++] = st;
                    }
                }
            }
        } else {
            int v = id - m->md.nfactors;
            r.kind = LEAF_UNITY;
            r.var = v;
            r.beta = pl.node[id].beta;
            auto it = std::find(m->slice_vars.begin(), m->slice_vars.end(), v);
            if (it != m->slice_vars.end()) r.slice_of_var = (int)(it - m->slice_vars.begin());
        }
        r.size = P.fwd[id].per;
        r.dst = P.fwd[id].off;
        r.mx = P.fwd[id].mx;
        P.leafrec.push_back(r);
    }
    P.nleafrec = n;
    // ---- descriptors and steps
    // per-tensor maxima: power-of-two scales (sum-product) or max-plus
    // normalisation offsets
    auto mxp = [&](int64_t i) { return P.mx + i; };
    auto fptr = [&](int id) { return (char *)P.arena + P.fwd[id].off * P.esz; };
    auto aptr = [&](int id) { return (char *)P.arena + P.adj[id].off * P.esz; };
    // forward tensors as the backward pass reads them (dropped ones from
    // their recompute slots)
    auto bfptr = [&](int id) {
        return P.drop[id] ? (char *)P.arena + P.rec_off[id] * P.esz : fptr(id);
    };
    const int store_t = dtype == 0 ? E_F64 : E_F32;
    size_t scratch = 0, need_x = 0, need_y = 0, need_d = 0;
    auto add_gemm = [&](std::vector<Step> &steps, const Opnd &X, const Opnd &Y, const Labels &bt,
                        const Labels &rows, const Labels &cols, const Labels &red,
                        const Labels &out_lab, bool out_beta, void *out_ptr,
                        unsigned long long *out_mx, double flops, double bytes) -> std::string {
        Step st;
        st.kind = 1;
        size_t nx, ny, nd2;
        std::string e = make_gemm_op(net.card, nbeta, store_t, P.gemm_type, X, Y, bt, rows, cols,
                                     red, out_lab, out_beta, out_ptr, out_mx, st.g, nx, ny, nd2);
        if (!e.empty()) return e;
        st.g.tc = use_tc;
        need_x = std::max(need_x, nx);
        need_y = std::max(need_y, ny);
        need_d = std::max(need_d, nd2);
        st.flops = flops;
        st.bytes = bytes;
        steps.push_back(st);
        return "";
    };
    auto per_items = [&](bool b) { return b ? (double)nbeta : 1.0; };
    // the forward step of node id writing its result at `outp` (the arena
    // slot, or the recompute slot of a dropped tensor); the operands are
    // always read from their forward slots
    auto fwd_step = [&](int id, char *outp, std::vector<Step> &steps, bool recomp,
                        bool record_desc) -> tn_status {
        const Node &nd = pl.node[id];
        CDesc d;
        err = make_desc(net.card, pl.node[nd.a].labels, pl.node[nd.a].beta, P.fwd[nd.a].per,
                        fptr(nd.a), mxp(P.fwd[nd.a].mx), pl.node[nd.b].labels, pl.node[nd.b].beta,
                        P.fwd[nd.b].per, fptr(nd.b), mxp(P.fwd[nd.b].mx), nd.labels, nd.beta,
                        outp, mxp(P.fwd[id].mx), &nd.elim, nbeta,
                        maxplus ? P.am + P.am_off[id] : nullptr, d);
        if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
        if (record_desc) P.fdesc.push_back(d);
        if (P.micro[id]) return TN_OK;
        double items = per_items(nd.beta);
        double flops = 2.0 * nd.muladds * items;
        double bytes = (double)P.esz * (P.fwd[nd.a].elems + P.fwd[nd.b].elems + P.fwd[id].elems);
        if (nd.gemm) {
            Opnd X{&pl.node[nd.ga].labels, pl.node[nd.ga].beta, P.fwd[nd.ga].per, fptr(nd.ga),
                   P.mx + P.fwd[nd.ga].mx};
            Opnd Y{&pl.node[nd.gb].labels, pl.node[nd.gb].beta, P.fwd[nd.gb].per, fptr(nd.gb),
                   P.mx + P.fwd[nd.gb].mx};
            err = add_gemm(steps, X, Y, nd.gbt, nd.gm, nd.gn, nd.elim, nd.labels, nd.beta,
                           outp, P.mx + P.fwd[id].mx, flops, bytes);
            if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
            steps.back().node = id;
            steps.back().recompute = recomp;
        } else {
            Step st;
            st.semiring = maxplus ? MAXPLUS : SUM;
            st.flops = flops;
            st.bytes = bytes;
            const Node &na = pl.node[nd.a], &nb = pl.node[nd.b];
            absorb_reject = "";
            if (make_absorb(net.card, na.labels, na.beta, P.fwd[nd.a].per, fptr(nd.a),
                            mxp(P.fwd[nd.a].mx), nb.labels, nb.beta, P.fwd[nd.b].per, fptr(nd.b),
                            mxp(P.fwd[nd.b].mx), nd.labels, nd.beta, P.fwd[id].per, outp,
                            mxp(P.fwd[id].mx), &nd.elim, nbeta,
                            maxplus ? P.am + P.am_off[id] : nullptr, st.ad, !maxplus) ||
                ((st.why = absorb_reject), false) ||
                make_absorb(net.card, nb.labels, nb.beta, P.fwd[nd.b].per, fptr(nd.b),
                            mxp(P.fwd[nd.b].mx), na.labels, na.beta, P.fwd[nd.a].per, fptr(nd.a),
                            mxp(P.fwd[nd.a].mx), nd.labels, nd.beta, P.fwd[id].per, outp,
                            mxp(P.fwd[id].mx), &nd.elim, nbeta,
                            maxplus ? P.am + P.am_off[id] : nullptr, st.ad, !maxplus)) {
                st.kind = 2;
            } else if (!maxplus &&
                       make_reduce(net.card, na.labels, na.beta, P.fwd[nd.a].per, fptr(nd.a),
                                   mxp(P.fwd[nd.a].mx), nb.labels, nb.beta, P.fwd[nd.b].per,
                                   fptr(nd.b), mxp(P.fwd[nd.b].mx), nd.labels, nd.beta,
                                   P.fwd[id].per, outp, mxp(P.fwd[id].mx), nbeta, st.rd) &&
                       st.rd.nm >= 4096) {
                st.kind = 3;
                scratch = std::max(scratch, reduce_scratch_bytes(st.rd, P.esz));
            } else if (!maxplus &&
                       make_bgemm(net.card, na.labels, na.beta, P.fwd[nd.a].per, fptr(nd.a),
                                  mxp(P.fwd[nd.a].mx), nb.labels, nb.beta, P.fwd[nd.b].per,
                                  fptr(nd.b), mxp(P.fwd[nd.b].mx), nd.labels, nd.beta,
                                  P.fwd[id].per, outp, mxp(P.fwd[id].mx), nbeta, P.esz, st.bd,
                                  st.btab)) {
                st.kind = 4;
                scratch = std::max(scratch, bgemm_scratch_bytes(st.bd, P.esz));
            } else {
                st.kind = 0;
                st.d = d;
                scratch = std::max(scratch, contract_scratch_bytes(d, P.esz));
            }
            st.node = id;
            st.recompute = recomp;
            steps.push_back(st);
        }
        return TN_OK;
    };
    for (int id = n; id < NN; ++id) {
        tn_status fs = fwd_step(id, fptr(id), P.fsteps, false, true);
        if (fs) return fs;
    }
    // label order of each adjoint tensor: the node's own, except where a
    // GEMM-form adjoint step can write its result straight from the GEMM
    // ([batch][rows][cols], no scatter pass); leaves and micro subtrees keep
    // the node order (marginals and the micro kernel read them so)
    std::vector<Labels> adjlab(NN);
    for (int i = 0; i < NN; ++i) adjlab[i] = pl.node[i].labels;
    auto alab = [&](int i) -> const Labels & { return adjlab[i]; };
    auto gemm_adj_layout = [&](int child, const Labels &bt, const Labels &rows,
                               const Labels &cols, bool xbeta, bool ybeta) {
        if (child < n || P.micro[child]) return;
        const int bpos = xbeta && ybeta ? 1 : xbeta ? 2 : ybeta ? 3 : 0;
        if (bpos == 3 || (bpos == 2 && !bt.empty())) return;   // batch label outermost
        Labels l(bt);
        l.insert(l.end(), rows.begin(), rows.end());
        l.insert(l.end(), cols.begin(), cols.end());
        adjlab[child] = l;
    };
    if (backward) {
        for (int id = NN - 1; id >= n; --id) {
            if (P.micro[id]) continue;
            const Node &nd = pl.node[id];
            const Node &na = pl.node[nd.a], &nb = pl.node[nd.b];
            char *cbar = aptr(id);
            for (int c : {nd.a, nd.b})
                if (P.drop[c] && P.rec_off[c] >= 0) {
                    tn_status rs = fwd_step(c, bfptr(c), P.bsteps, true, false);
                    if (rs) return rs;
                }
            double items = per_items(P.adj_beta[id]);
            double flops = 2.0 * nd.muladds * items;
            if (nd.gemm) {
                const Node &xa = pl.node[nd.ga], &xb = pl.node[nd.gb];
                Opnd Cb{&alab(id), (bool)P.adj_beta[id], P.adj[id].per, cbar, P.mx + P.adj[id].mx};
                Opnd A{&xa.labels, xa.beta, P.fwd[nd.ga].per, bfptr(nd.ga), P.mx + P.fwd[nd.ga].mx};
                Opnd Bo{&xb.labels, xb.beta, P.fwd[nd.gb].per, bfptr(nd.gb), P.mx + P.fwd[nd.gb].mx};
                if (P.need_adj[nd.ga]) {
                    // Abar[bt, m, k] = sum_n Cbar[bt, m, n] B[bt, k, n]
                    gemm_adj_layout(nd.ga, nd.gbt, nd.gm, nd.elim, P.adj_beta[id], xb.beta);
                    double bytes = (double)P.esz * (P.adj[id].elems + P.fwd[nd.gb].elems +
                                                    P.adj[nd.ga].elems);
                    err = add_gemm(P.bsteps, Cb, Bo, nd.gbt, nd.gm, nd.elim, nd.gn, alab(nd.ga),
                                   P.adj_beta[nd.ga], aptr(nd.ga), P.mx + P.adj[nd.ga].mx, flops,
                                   bytes);
                    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                    P.bsteps.back().node = nd.ga;
                    P.bsteps.back().adjoint = true;
                }
                if (P.need_adj[nd.gb]) {
                    // Bbar[bt, k, n] = sum_m A[bt, m, k] Cbar[bt, m, n]
                    gemm_adj_layout(nd.gb, nd.gbt, nd.elim, nd.gn, xa.beta, P.adj_beta[id]);
                    double bytes = (double)P.esz * (P.fwd[nd.ga].elems + P.adj[id].elems +
                                                    P.adj[nd.gb].elems);
                    err = add_gemm(P.bsteps, A, Cb, nd.gbt, nd.elim, nd.gn, nd.gm, alab(nd.gb),
                                   P.adj_beta[nd.gb], aptr(nd.gb), P.mx + P.adj[nd.gb].mx, flops,
                                   bytes);
                    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                    P.bsteps.back().node = nd.gb;
                    P.bsteps.back().adjoint = true;
                }
                continue;
            }
            if (P.need_adj[nd.a]) {
                // Abar = con(Cbar, B -> Va): stream Cbar once, B small
                Step st;
                st.flops = flops;
                st.bytes = (double)P.esz * (P.adj[id].elems + P.fwd[nd.b].elems + P.adj[nd.a].elems);
                if (make_absorb(net.card, alab(id), P.adj_beta[id], P.adj[id].per, cbar,
                                P.mx + P.adj[id].mx, nb.labels, nb.beta, P.fwd[nd.b].per,
                                bfptr(nd.b), P.mx + P.fwd[nd.b].mx, alab(nd.a), P.adj_beta[nd.a],
                                P.adj[nd.a].per, aptr(nd.a), P.mx + P.adj[nd.a].mx, nullptr, nbeta,
                                nullptr, st.ad, true) ||
                    make_absorb(net.card, nb.labels, nb.beta, P.fwd[nd.b].per, bfptr(nd.b),
                                P.mx + P.fwd[nd.b].mx, alab(id), P.adj_beta[id], P.adj[id].per,
                                cbar, P.mx + P.adj[id].mx, alab(nd.a), P.adj_beta[nd.a],
                                P.adj[nd.a].per, aptr(nd.a), P.mx + P.adj[nd.a].mx, nullptr, nbeta,
                                nullptr, st.ad, true)) {
                    st.kind = 2;
                } else if (make_bgemm(net.card, alab(id), P.adj_beta[id], P.adj[id].per, cbar,
                                      P.mx + P.adj[id].mx, nb.labels, nb.beta, P.fwd[nd.b].per,
                                      bfptr(nd.b), P.mx + P.fwd[nd.b].mx, alab(nd.a),
                                      P.adj_beta[nd.a], P.adj[nd.a].per, aptr(nd.a),
                                      P.mx + P.adj[nd.a].mx, nbeta, P.esz, st.bd, st.btab)) {
                    st.kind = 4;
                    scratch = std::max(scratch, bgemm_scratch_bytes(st.bd, P.esz));
                } else {
                    err = make_desc(net.card, alab(id), P.adj_beta[id], P.adj[id].per, cbar,
                                    P.mx + P.adj[id].mx, nb.labels, nb.beta, P.fwd[nd.b].per,
                                    bfptr(nd.b), P.mx + P.fwd[nd.b].mx, alab(nd.a), P.adj_beta[nd.a],
                                    aptr(nd.a), P.mx + P.adj[nd.a].mx, nullptr, nbeta, nullptr,
                                    st.d);
                    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                    st.kind = 0;
                    st.why = absorb_reject;
                    scratch = std::max(scratch, contract_scratch_bytes(st.d, P.esz));
                }
                st.node = nd.a;
                st.adjoint = true;
                P.bsteps.push_back(st);
            }
            if (P.need_adj[nd.b]) {
                // Bbar = con(A, Cbar -> Vb): stream A and Cbar once, Bbar small
                Step st;
                st.flops = flops;
                st.bytes = (double)P.esz * (P.fwd[nd.a].elems + P.adj[id].elems + P.adj[nd.b].elems);
                if (P.adj[nd.b].elems >= (1 << 16) &&
                    (make_absorb(net.card, na.labels, na.beta, P.fwd[nd.a].per, bfptr(nd.a),
                                 P.mx + P.fwd[nd.a].mx, alab(id), P.adj_beta[id], P.adj[id].per,
                                 cbar, P.mx + P.adj[id].mx, alab(nd.b), P.adj_beta[nd.b],
                                 P.adj[nd.b].per, aptr(nd.b), P.mx + P.adj[nd.b].mx, nullptr,
                                 nbeta, nullptr, st.ad, true) ||
                     make_absorb(net.card, alab(id), P.adj_beta[id], P.adj[id].per, cbar,
                                 P.mx + P.adj[id].mx, na.labels, na.beta, P.fwd[nd.a].per,
                                 bfptr(nd.a), P.mx + P.fwd[nd.a].mx, alab(nd.b), P.adj_beta[nd.b],
                                 P.adj[nd.b].per, aptr(nd.b), P.mx + P.adj[nd.b].mx, nullptr,
                                 nbeta, nullptr, st.ad, true))) {
                    st.kind = 2;
                } else if (make_reduce(net.card, na.labels, na.beta, P.fwd[nd.a].per, bfptr(nd.a),
                                P.mx + P.fwd[nd.a].mx, alab(id), P.adj_beta[id], P.adj[id].per,
                                cbar, P.mx + P.adj[id].mx, alab(nd.b), P.adj_beta[nd.b],
                                P.adj[nd.b].per, aptr(nd.b), P.mx + P.adj[nd.b].mx, nbeta, st.rd) &&
                    st.rd.nm >= 4096) {
                    st.kind = 3;
                    scratch = std::max(scratch, reduce_scratch_bytes(st.rd, P.esz));
                } else if (make_bgemm(net.card, na.labels, na.beta, P.fwd[nd.a].per, bfptr(nd.a),
                                      P.mx + P.fwd[nd.a].mx, alab(id), P.adj_beta[id],
                                      P.adj[id].per, cbar, P.mx + P.adj[id].mx, alab(nd.b),
                                      P.adj_beta[nd.b], P.adj[nd.b].per, aptr(nd.b),
                                      P.mx + P.adj[nd.b].mx, nbeta, P.esz, st.bd, st.btab)) {
                    st.kind = 4;
                    scratch = std::max(scratch, bgemm_scratch_bytes(st.bd, P.esz));
                } else {
                    err = make_desc(net.card, na.labels, na.beta, P.fwd[nd.a].per, bfptr(nd.a),
                                    P.mx + P.fwd[nd.a].mx, alab(id), P.adj_beta[id], P.adj[id].per,
                                    cbar, P.mx + P.adj[id].mx, alab(nd.b), P.adj_beta[nd.b],
                                    aptr(nd.b), P.mx + P.adj[nd.b].mx, nullptr, nbeta, nullptr,
                                    st.d);
                    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                    st.kind = 0;
                    st.why = absorb_reject;
                    scratch = std::max(scratch, contract_scratch_bytes(st.d, P.esz));
                }
                st.node = nd.b;
                st.adjoint = true;
                P.bsteps.push_back(st);
            }
        }
    }
    // micro lists, grouped by the lane of their subtree (each lane runs its
    // own subtrees first in the forward pass and last in the backward pass)
    std::vector<std::pair<int, int>> morder;   // (lane, micro root)
    for (auto &kv : msub) morder.push_back({P.lane[kv.first], kv.first});
    std::stable_sort(morder.begin(), morder.end(),
                     [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
                         return x.first < y.first;
                     });
    P.mlane_beg.assign(P.nlanes + 1, 0);
    for (auto &lo : morder) P.mlane_beg[lo.first + 1]++;
    for (int l = 0; l < P.nlanes; ++l) P.mlane_beg[l + 1] += P.mlane_beg[l];
    for (auto &lo : morder) {
        auto &kv = *msub.find(lo.second);
        P.mf_beg.push_back((int32_t)P.mf.size());
        for (int id : kv.second) {
            MicroDesc md;
            if (!to_micro(P.fdesc[id - n], P.arena, P.esz, P.mx, P.am, md))
                return fail(TN_E_UNSUPPORTED, "micro node conversion");
            P.mf.push_back(md);
        }
        if (!backward) continue;
        P.mb_beg.push_back((int32_t)P.mb.size());
        for (auto it = kv.second.rbegin(); it != kv.second.rend(); ++it) {
            int id = *it;
            const Node &nd = pl.node[id];
            const Node &na = pl.node[nd.a], &nb = pl.node[nd.b];
            char *cbar = aptr(id);
            CDesc d;
            MicroDesc md;
            if (P.need_adj[nd.a]) {
                err = make_desc(net.card, alab(id), P.adj_beta[id], P.adj[id].per, cbar,
                                P.mx + P.adj[id].mx, nb.labels, nb.beta, P.fwd[nd.b].per,
                                fptr(nd.b), P.mx + P.fwd[nd.b].mx, alab(nd.a), P.adj_beta[nd.a],
                                aptr(nd.a), P.mx + P.adj[nd.a].mx, nullptr, nbeta, nullptr, d);
                if (!err.empty() || !to_micro(d, P.arena, P.esz, P.mx, P.am, md))
                    return fail(TN_E_UNSUPPORTED, "micro adjoint conversion");
                P.mb.push_back(md);
            }
            if (P.need_adj[nd.b]) {
                err = make_desc(net.card, na.labels, na.beta, P.fwd[nd.a].per, fptr(nd.a),
                                P.mx + P.fwd[nd.a].mx, alab(id), P.adj_beta[id], P.adj[id].per,
                                cbar, P.mx + P.adj[id].mx, alab(nd.b), P.adj_beta[nd.b],
                                aptr(nd.b), P.mx + P.adj[nd.b].mx, nullptr, nbeta, nullptr, d);
                if (!err.empty() || !to_micro(d, P.arena, P.esz, P.mx, P.am, md))
                    return fail(TN_E_UNSUPPORTED, "micro adjoint conversion");
                P.mb.push_back(md);
            }
        }
    }
    P.mf_beg.push_back((int32_t)P.mf.size());
    P.mb_beg.push_back((int32_t)P.mb.size());
    if (!P.mf.empty()) {
        CK(P.mem.alloc(&P.d_mf, sizeof(MicroDesc) * P.mf.size()));
        CK(cudaMemcpy(P.d_mf, P.mf.data(), sizeof(MicroDesc) * P.mf.size(), cudaMemcpyHostToDevice));
        CK(P.mem.alloc(&P.d_mf_beg, 4 * P.mf_beg.size()));
        CK(cudaMemcpy(P.d_mf_beg, P.mf_beg.data(), 4 * P.mf_beg.size(), cudaMemcpyHostToDevice));
    }
    if (!P.mb.empty()) {
        CK(P.mem.alloc(&P.d_mb, sizeof(MicroDesc) * P.mb.size()));
        CK(cudaMemcpy(P.d_mb, P.mb.data(), sizeof(MicroDesc) * P.mb.size(), cudaMemcpyHostToDevice));
        CK(P.mem.alloc(&P.d_mb_beg, 4 * P.mb_beg.size()));
        CK(cudaMemcpy(P.d_mb_beg, P.mb_beg.data(), 4 * P.mb_beg.size(), cudaMemcpyHostToDevice));
    }
    // ---- step lanes and the events that order them across lanes: event id
    // for fwd[v] = v, for adj[v] = NN + v (the root adjoint's is recorded
    // after it is set to one), 2 NN = start, 2 NN + 1 + l = end of lane l
    {
        std::vector<int> prod_f(NN, -1), prod_b(NN, -1);
        for (int i = 0; i < (int)P.fsteps.size(); ++i) {
            Step &st = P.fsteps[i];
            st.lane = st.node >= 0 ? P.lane[st.node] : 0;
            if (st.node >= 0) prod_f[st.node] = i;
        }
        for (int i = 0; i < (int)P.bsteps.size(); ++i) {
            Step &st = P.bsteps[i];
            st.lane = st.node >= 0 ? P.lane[st.node] : 0;
            if (st.node >= 0) prod_b[st.node] = i;
        }
        if (P.nlanes > 1) {
            for (auto &st : P.fsteps) {
                if (st.node < 0) continue;
                const Node &nd = pl.node[st.node];
                for (int c : {nd.a, nd.b})
                    if (c >= n && !P.micro[c] && P.lane[c] != st.lane && prod_f[c] >= 0) {
                        st.waits.push_back(c);
                        P.fsteps[prod_f[c]].rec = c;
                    }
            }
            for (auto &st : P.bsteps) {
                if (st.node < 0) continue;
                const int par = pl.node[st.node].parent;
                if (par < 0 || P.lane[par] == st.lane) continue;
                st.waits.push_back(NN + par);
                if (par != pl.root && prod_b[par] >= 0) P.bsteps[prod_b[par]].rec = NN + par;
            }
        }
    }
    for (auto *steps : {&P.fsteps, &P.bsteps})
        for (auto &st : *steps) {
            if (st.kind == 2) st.ad.bps = P.tune.absorb_bps;
            if (st.kind == 4) {
                st.bd.err = m->d_err;
                // programs keep the FP32 CUDA-core form: in the evidence-
                // batched tree the persistent tensor-core gather kernel (one
                // CTA per SM) measured slower (it holds every SM against the
                // other lanes of the graph) and its TF32 inputs raised the
                // log Z error; tn_contract_dev uses it for TF32 / BF16
                st.bd.tc = 0;
            }
        }
    // inner offset tables of the streaming steps, one device buffer
    {
        std::vector<int32_t> all, t;
        std::vector<std::pair<Step *, size_t>> where;
        std::vector<std::pair<PDesc *, size_t>> pwhere;
        for (auto *steps : {&P.fsteps, &P.bsteps})
            for (auto &st : *steps) {
                if (st.kind == 1) {
                    GemmOp &g = st.g;
                    for (auto pr : {std::make_pair(&g.px, &g.tpx), std::make_pair(&g.py, &g.tpy),
                                    std::make_pair(&g.post, &g.tpost)}) {
                        if (pr.first->tl.tn <= 0) continue;
                        all.resize((all.size() + 3) & ~(size_t)3);   // 16-byte aligned
                        pwhere.push_back({pr.first, all.size()});
                        all.insert(all.end(), pr.second->begin(), pr.second->end());
                    }
                    continue;
                }
                if (st.kind == 2) absorb_table(st.ad, P.esz, t);
                else if (st.kind == 3) reduce_table(st.rd, P.esz, t);
                else if (st.kind == 4) t = st.btab;
                else continue;
                all.resize((all.size() + 3) & ~(size_t)3);   // 16-byte aligned
                where.push_back({&st, all.size()});
                all.insert(all.end(), t.begin(), t.end());
            }
        if (!all.empty()) {
            int32_t *dt = nullptr;
            CK(P.mem.alloc(&dt, all.size() * 4));
            CK(cudaMemcpy(dt, all.data(), all.size() * 4, cudaMemcpyHostToDevice));
            for (auto &w : where) {
                if (w.first->kind == 2) w.first->ad.tab = dt + w.second;
                else if (w.first->kind == 3) w.first->rd.tab = dt + w.second;
                else {
                    BDesc &b = w.first->bd;
                    const int32_t *base = dt + w.second;
                    for (const int32_t **q : {&b.tag, &b.tbg, &b.tcg, &b.tam, &b.tcm, &b.tbn,
                                              &b.tcn, &b.tak, &b.tbk})
                        *q = base + (intptr_t)*q;
                    if (getenv("TN_PLAN_TRACE") && getenv("TN_PLAN_TRACE")[0] == '1') {
                        // plan trace: the first offsets of each group table
                        const std::vector<int32_t> &t = w.first->btab;
                        const int64_t sz[9] = {b.G, b.G, b.G, b.M, b.M, b.N, b.N, b.K, b.K};
                        const char *nm[9] = {"ag", "bg", "cg", "am", "cm", "bn", "cn", "ak", "bk"};
                        int64_t at = 0;
                        fprintf(stderr, "bgemm tables G %lld M %lld N %lld K %lld:",
                                (long long)b.G, (long long)b.M, (long long)b.N, (long long)b.K);
                        for (int q = 0; q < 9; ++q) {
                            fprintf(stderr, " %s", nm[q]);
                            for (int64_t i = 0; i < std::min<int64_t>(sz[q], 8); ++i)
                                fprintf(stderr, ",%d", t[at + i]);
                            at += sz[q];
                        }
                        fprintf(stderr, "\n");
                    }
                    w.first->btab.clear();
                    w.first->btab.shrink_to_fit();
                }
            }
            for (auto &w : pwhere) w.first->tl.ttab = dt + w.second;
        }
    }
    trace_program(P);
    // GEMM workspaces (one set per lane that runs GEMM steps), then patch
    // the steps' workspace pointers
    {
        std::vector<char> has_gemm(P.nlanes, 0);
        for (auto *steps : {&P.fsteps, &P.bsteps})
            for (auto &st : *steps)
                if (st.kind == 1) has_gemm[st.lane] = 1;
        std::vector<std::array<char *, 3>> ws(P.nlanes, {nullptr, nullptr, nullptr});
        for (int l = 0; l < P.nlanes; ++l) {
            if (!has_gemm[l]) continue;
            if (need_x) CK(P.mem.alloc(&ws[l][0], need_x));
            if (need_y) CK(P.mem.alloc(&ws[l][1], need_y));
            if (need_d) CK(P.mem.alloc(&ws[l][2], need_d));
        }
        P.wsX = ws[0][0];
        P.wsY = ws[0][1];
        P.wsD = ws[0][2];
        for (auto *steps : {&P.fsteps, &P.bsteps})
            for (auto &st : *steps) {
                if (st.kind != 1) continue;
                char *wx = ws[st.lane][0], *wy = ws[st.lane][1], *wd = ws[st.lane][2];
                st.g.px.out = wx;
                st.g.py.out = wy;
                if (!st.g.x_in_place) st.g.g.X = wx;
                st.g.g.Y = wy;
                if (st.g.has_post) {
                    st.g.g.D = wd;
                    st.g.post.in = wd;
                }
                st.g.tc = st.g.tc && tc_gemm_supported(st.g.g);
            }
    }
    P.scratch_bytes = scratch;
    P.lscratch.assign(P.nlanes, nullptr);
    if (scratch)
        for (int l = 0; l < P.nlanes; ++l) CK(P.mem.alloc(&P.lscratch[l], scratch));
    P.scratch = P.lscratch[0];
    // completion counters of the reduce steps (one per group and item)
    P.nrcnt = 0;
    for (auto *steps : {&P.fsteps, &P.bsteps})
        for (auto &st : *steps)
            if (st.kind == 3) P.nrcnt = std::max<int64_t>(P.nrcnt, st.rd.ng * st.rd.nbeta);
    if (P.nrcnt) {
        // one counter set per lane, contiguous so that one memset clears all
        CK(P.mem.alloc(&P.rcnt, (size_t)P.nrcnt * P.nlanes * 4));
        CK(cudaMemset(P.rcnt, 0, (size_t)P.nrcnt * P.nlanes * 4));
        for (auto *steps : {&P.fsteps, &P.bsteps})
            for (auto &st : *steps)
                if (st.kind == 3) st.rd.cnt = P.rcnt + (size_t)st.lane * P.nrcnt;
    }
    // ---- leaf records to device
    CK(P.mem.alloc(&P.d_leaf, sizeof(LeafRec) * n));
    CK(cudaMemcpy(P.d_leaf, P.leafrec.data(), sizeof(LeafRec) * n, cudaMemcpyHostToDevice));
    // ---- exponent (sum-product) or offset (max-plus) list for log Z
    {
        std::vector<int64_t> ex;
        for (int id = 0; id < NN; ++id) {
            if (id == pl.root) continue;
            ex.push_back(P.fwd[id].mx);
            ex.push_back(P.fwd[id].beta ? 1 : 0);
        }
        P.nexps = (int)(ex.size() / 2);
        CK(P.mem.alloc(&P.d_exps, ex.size() * 8));
        CK(cudaMemcpy(P.d_exps, ex.data(), ex.size() * 8, cudaMemcpyHostToDevice));
    }
    // ---- marginal / gradient records
    if (backward) {
        std::vector<MargRec> mr;
        int64_t moff = 0;
        for (int v = 0; v < m->md.nvars; ++v) {
            int id = m->md.nfactors + v;
            MargRec r;
            std::memset(&r, 0, sizeof r);
            r.fwd = P.fwd[id].off;
            r.adj = P.adj[id].off;
            r.moff = moff;
            r.card = m->md.card[v];
            r.fbeta = P.fwd[id].beta;
            r.abeta = P.adj_beta[id];
            r.sliced = std::find(m->slice_vars.begin(), m->slice_vars.end(), v) !=
                       m->slice_vars.end();
            moff += r.card;
            mr.push_back(r);
        }
        P.marg_stride = moff;
        CK(P.mem.alloc(&P.d_margrec, sizeof(MargRec) * std::max<size_t>(1, mr.size())));
        if (!mr.empty())
            CK(cudaMemcpy(P.d_margrec, mr.data(), sizeof(MargRec) * mr.size(),
                          cudaMemcpyHostToDevice));
        CK(P.mem.alloc(&P.d_marg, (size_t)nbeta * std::max<int64_t>(1, moff) * 8));
        if (grads) {
            std::vector<GradRec> gr;
            for (int f = 0; f < m->md.nfactors; ++f) {
                GradRec r;
                std::memset(&r, 0, sizeof r);
                r.fwd = P.fwd[f].off;
                r.adj = P.adj[f].off;
                r.size = P.fwd[f].per;
                r.goff = m->md.toff[f];
                r.abeta = P.adj_beta[f];
                gr.push_back(r);
            }
            P.ngrad = (int)gr.size();
            P.grad_stride = (int64_t)m->md.tables.size();
            CK(P.mem.alloc(&P.d_gradrec, sizeof(GradRec) * std::max<size_t>(1, gr.size())));
            if (!gr.empty())
                CK(cudaMemcpy(P.d_gradrec, gr.data(), sizeof(GradRec) * gr.size(),
                              cudaMemcpyHostToDevice));
            CK(P.mem.alloc(&P.d_grad, (size_t)nbeta * std::max<int64_t>(1, P.grad_stride) * 8));
        }
    }
    // ---- backtrack records (root first)
    if (maxplus) {
        std::vector<int64_t> meta;
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            meta.push_back((int64_t)nd.labels.size());
            for (int v : nd.labels) {
                meta.push_back(v);
                meta.push_back(stride_in(net.card, nd.labels, v));
            }
            meta.push_back((int64_t)nd.elim.size());
            for (int v : nd.elim) {
                meta.push_back(v);
                meta.push_back(net.card[v]);
            }
            meta.push_back(P.am_off[id]);
            meta.push_back(P.fwd[id].per);
            meta.push_back(P.fwd[id].beta ? 1 : 0);
        }
        P.nmeta = NN - n;
        CK(P.mem.alloc(&P.d_meta, meta.size() * 8));
        CK(cudaMemcpy(P.d_meta, meta.data(), meta.size() * 8, cudaMemcpyHostToDevice));
        CK(P.mem.alloc(&P.d_assign, (size_t)nbeta * std::max(1, (int)net.card.size()) * 4));
    }
    // ---- sampling records (root first)
    if (kind == K_SAMPLE) {
        std::vector<int64_t> meta;
        int64_t cdf_total = 0;
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            const Node &na = pl.node[nd.a], &nb = pl.node[nd.b];
            meta.push_back((int64_t)nd.labels.size());
            for (int v : nd.labels) {
                meta.push_back(v);
                meta.push_back(std::max<int64_t>(0, stride_in(net.card, na.labels, v)));
                meta.push_back(std::max<int64_t>(0, stride_in(net.card, nb.labels, v)));
                meta.push_back(stride_in(net.card, nd.labels, v));
            }
            int64_t K = 1;
            meta.push_back((int64_t)nd.elim.size());
            for (int v : nd.elim) {
                meta.push_back(v);
                meta.push_back(net.card[v]);
                meta.push_back(std::max<int64_t>(0, stride_in(net.card, na.labels, v)));
                meta.push_back(std::max<int64_t>(0, stride_in(net.card, nb.labels, v)));
                K *= net.card[v];
            }
            meta.push_back(P.fwd[nd.a].off);
            meta.push_back(P.fwd[nd.b].off);
            meta.push_back(K);
            // large summed spaces get cumulative tables (binary search per
            // sample) while those fit 2^27 entries; otherwise every sample
            // scans the node's summed space directly
            const int64_t rows = P.fwd[id].per;
            if (K > 4096 && (double)rows * (double)K <= (double)(1LL << 27)) {
                meta.push_back(cdf_total);
                P.cdf_nodes.push_back({P.fdesc[id - n], rows});
                cdf_total += rows * K;
            } else {
                meta.push_back(-1);
            }
        }
        P.nmeta = NN - n;
        CK(P.mem.alloc(&P.d_meta, meta.size() * 8));
        CK(cudaMemcpy(P.d_meta, meta.data(), meta.size() * 8, cudaMemcpyHostToDevice));
        if (cdf_total) CK(P.mem.alloc(&P.cdf, (size_t)cdf_total * 8));
    }
    return TN_OK;
}

// Per-class device time accumulated by a profiling run.  Every launch is
// bracketed by a pair of events recorded back to back on the stream (no host
// synchronisation between launches, so the device runs them as in a graph
// replay); the durations are read once the run has finished.
struct Prof {
    double ms[C_NCLS] = {0};
    double n[C_NCLS] = {0};
    double flops[C_NCLS] = {0};
    double bytes[C_NCLS] = {0};
    std::vector<cudaEvent_t> ev;     // start, end per launch
    std::vector<double> meta;        // per launch: class, flops, bytes
    std::vector<double> rec;         // per launch: class, ms, flops, bytes
    ~Prof() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    void finish() {
        for (size_t i = 0; i < meta.size() / 3; ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            int cls = (int)meta[3 * i];
            this->ms[cls] += ms;
            n[cls] += 1;
            flops[cls] += meta[3 * i + 1];
            bytes[cls] += meta[3 * i + 2];
            rec.insert(rec.end(), {(double)cls, (double)ms, meta[3 * i + 1], meta[3 * i + 2]});
        }
    }
};

template <typename F>
static void timed(Prof *pr, cudaStream_t st, int cls, double flops, double bytes, F &&f) {
    if (!pr) {
        f();
        return;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pr->ev.push_back(e0);
    pr->ev.push_back(e1);
    cudaEventRecord(e0, st);
    f();
    cudaEventRecord(e1, st);
    pr->meta.insert(pr->meta.end(), {(double)cls, flops, bytes});
}

template <typename T>
static void run_step(tn_model *m, Program &P, const Step &s, cudaStream_t st, int &nl, Prof *pr) {
    // recompute steps are profiled as their own class (not algorithmic work)
    auto cls = [&](int c) { return s.recompute ? (int)C_RECOMP : c; };
    if (s.kind == 2) {
        timed(pr, st, cls(C_STREAM), s.flops, s.bytes, [&] { launch_absorb<T>(s.ad, s.semiring, st); });
        ++nl;
        return;
    }
    if (s.kind == 3) {
        timed(pr, st, cls(C_SPLITK), s.flops, s.bytes,
              [&] { launch_reduce<T>(s.rd, P.lscratch[s.lane], st); });
        nl += reduce_launches(s.rd);
        return;
    }
    if (s.kind == 4) {
        timed(pr, st, cls(C_BGEMM), s.flops, s.bytes,
              [&] { launch_bgemm<T>(s.bd, P.lscratch[s.lane], st); });
        nl += bgemm_launches(s.bd);
        return;
    }
    if (s.kind == 0) {
        int c = cls(contract_uses_splitk(s.d) ? C_SPLITK : C_GENERIC);
        timed(pr, st, c, s.flops, s.bytes, [&] {
            launch_contract<T>(s.d, s.semiring, P.lscratch[s.lane], P.scratch_bytes, st, &nl);
        });
        return;
    }
    const GemmOp &g = s.g;
    timed(pr, st, cls(C_PREP), 0, g.prep_bytes, [&] {
        if (!g.x_in_place) launch_permute(g.px, st);
        launch_permute(g.py, st);
    });
    nl += g.x_in_place ? 1 : 2;
    if (g.tc) {
        timed(pr, st, cls(C_TCGEMM), s.flops, s.bytes, [&] { launch_tc_gemm(g.g, m->d_err, st); });
    } else {
        timed(pr, st, cls(C_SIMTGEMM), s.flops, s.bytes, [&] { launch_simt_gemm(g.g, st); });
    }
    ++nl;
    if (g.has_post) {
        timed(pr, st, cls(C_PREP), 0, g.post_bytes, [&] { launch_permute(g.post, st); });
        ++nl;
    }
}

// `lanes` (capture only): the streams of lanes 1 .. nlanes-1; without them
// every step runs in order on `st`.
template <typename T>
void enqueue_program(tn_model *m, Program &P, cudaStream_t st, Prof *pr = nullptr,
                     const std::vector<cudaStream_t> *lanes = nullptr) {
    const Plan &pl = P.plan;
    const int n = pl.tree.nleaves, NN = 2 * n - 1;
    const bool maxplus = P.kind == K_MAP || P.kind == K_MAXNET;
    int nl = 0;
    cudaMemsetAsync(P.mx, 0, (size_t)P.nmx * 8, st);
    if (P.nrcnt) cudaMemsetAsync(P.rcnt, 0, (size_t)P.nrcnt * P.nlanes * 4, st);
    ++nl;
    launch_leaves<T>(P.d_leaf, P.nleafrec, m->d_tables, P.d_card, m->md.nvars, P.d_evid, P.nbeta,
                     maxplus ? 1 : 0, (T *)P.arena, P.mx, m->d_flags, P.d_slice_val, st);
    ++nl;
    const bool par = lanes && P.nlanes > 1 && (int)P.ev.size() >= 2 * NN + 1 + P.nlanes;
    auto lane_stream = [&](int l) { return (par && l > 0) ? (*lanes)[l - 1] : st; };
    if (par) {
        cudaEventRecord(P.ev[2 * NN], st);
        for (int l = 1; l < P.nlanes; ++l) cudaStreamWaitEvent(lane_stream(l), P.ev[2 * NN], 0);
    }
    // micro subtrees: one launch, or one per lane when the lanes run apart
    auto micro = [&](const MicroDesc *d, const int32_t *beg, int sem) {
        if (!par) {
            int ns = (int)P.mlane_beg.back();
            if (ns > 0) {
                timed(pr, st, C_SMALL, 0, 0,
                      [&] { launch_micro<T>(d, beg, ns, sem, (T *)P.arena, P.mx, P.am, st); });
                ++nl;
            }
            return;
        }
        for (int l = 0; l < P.nlanes; ++l) {
            int s0 = P.mlane_beg[l], s1 = P.mlane_beg[l + 1];
            if (s1 <= s0) continue;
            launch_micro<T>(d, beg + s0, s1 - s0, sem, (T *)P.arena, P.mx, P.am, lane_stream(l));
            ++nl;
        }
    };
    if (!P.mf.empty()) micro(P.d_mf, P.d_mf_beg, maxplus ? MAXPLUS : SUM);
    auto run_steps = [&](std::vector<Step> &steps) {
        for (auto &s : steps) {
            cudaStream_t ls = lane_stream(s.lane);
            if (par)
                for (int w : s.waits) cudaStreamWaitEvent(ls, P.ev[w], 0);
            run_step<T>(m, P, s, ls, nl, pr);
            if (par && s.rec >= 0) cudaEventRecord(P.ev[s.rec], ls);
        }
    };
    auto join_lanes = [&] {
        for (int l = 1; par && l < P.nlanes; ++l) {
            cudaEventRecord(P.ev[2 * NN + 1 + l], lane_stream(l));
            cudaStreamWaitEvent(st, P.ev[2 * NN + 1 + l], 0);
        }
    };
    run_steps(P.fsteps);
    if (P.kind != K_MAR) join_lanes();
    const Slot &rs = P.fwd[pl.root];
    if (P.kind != K_SUMNET && P.kind != K_MAXNET) {
        launch_logz<T>(P.nbeta, (const T *)P.arena + rs.off, rs.beta ? 1 : 0, P.mx, P.d_exps,
                       P.nexps, P.d_logz, P.d_sigma, maxplus ? 1 : 0, st);
        ++nl;
    } else if (!maxplus) {
        launch_logz<T>(P.nbeta, (const T *)P.arena + rs.off, rs.beta ? 1 : 0, P.mx, P.d_exps,
                       P.nexps, P.d_logz, P.d_sigma, 0, st);
        ++nl;
    }
    if (P.kind == K_MAR) {
        const Slot &ra = P.adj[pl.root];
        launch_fill_one<T>((T *)P.arena + ra.off, ra.elems, P.mx + ra.mx, st);
        ++nl;
        if (par) cudaEventRecord(P.ev[NN + pl.root], st);
        run_steps(P.bsteps);
        if (!P.mb.empty()) micro(P.d_mb, P.d_mb_beg, SUM);
        join_lanes();
        launch_marginals<T>(P.d_margrec, m->md.nvars, P.nbeta, (const T *)P.arena,
                            (const T *)P.arena, P.d_marg, P.marg_stride, st);
        ++nl;
        if (P.grads) {
            launch_factor_grads<T>(P.d_gradrec, P.ngrad, P.nbeta, (const T *)P.arena,
                                   (const T *)P.arena, P.d_grad, P.grad_stride, st);
            ++nl;
        }
    }
    if (maxplus && P.kind == K_MAP) {
        cudaMemcpyAsync(P.d_assign, P.d_evid, (size_t)P.nbeta * m->md.nvars * 4,
                        cudaMemcpyDeviceToDevice, st);
        launch_backtrack(P.d_meta, P.nmeta, P.am, P.nbeta, m->md.nvars, P.d_assign, st);
        ++nl;
    }
    (void)NN;
    P.launches = nl;
}

tn_status capture_program(tn_model *m, Program &P) {
    cudaGraph_t g = nullptr;
    if (P.nlanes > 1) {
        while ((int)m->lanes.size() < P.nlanes - 1) {
            cudaStream_t l;
            CK(cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking));
            m->lanes.push_back(l);
        }
        const int NN = 2 * P.plan.tree.nleaves - 1;
        while ((int)P.ev.size() < 2 * NN + 1 + P.nlanes) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            P.ev.push_back(e);
        }
    }
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    if (P.dtype == 0) enqueue_program<double>(m, P, m->stream, nullptr, &m->lanes);
    else enqueue_program<float>(m, P, m->stream, nullptr, &m->lanes);
    cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (e != cudaSuccess) return fail(TN_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&P.gexec, g, 0);
    P.graph = g;
    if (e != cudaSuccess) return fail(TN_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return TN_OK;
}

tn_status ensure_device(tn_model *m) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (m->device == dev && m->d_tables && !m->tables_overridden) return TN_OK;
    if (m->device != dev) {
        m->progs.clear();
        m->mmap.reset();
        if (m->d_tables) cudaFree(m->d_tables);
        m->d_tables = nullptr;
        if (m->stream) cudaStreamDestroy(m->stream);
        for (auto l : m->lanes) cudaStreamDestroy(l);
        m->lanes.clear();
        if (m->ev0) cudaEventDestroy(m->ev0);
        if (m->ev1) cudaEventDestroy(m->ev1);
        CK(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
        CK(cudaEventCreate(&m->ev0));
        CK(cudaEventCreate(&m->ev1));
        m->device = dev;
    }
    size_t tb = std::max<size_t>(8, m->md.tables.size() * 8);
    if (!m->d_tables) CK(cudaMalloc(&m->d_tables, tb));
    if (!m->d_flags) CK(cudaMalloc(&m->d_flags, 16));
    CK(cudaMemset(m->d_flags, 0, 16));
    if (!m->d_err) {
        CK(cudaMalloc(&m->d_err, 16));
        CK(cudaMemset(m->d_err, 0, 16));
    }
    if (!m->md.tables.empty())
        CK(cudaMemcpy(m->d_tables, m->md.tables.data(), m->md.tables.size() * 8,
                      cudaMemcpyHostToDevice));
    m->tables_overridden = false;
    return TN_OK;
}

int dtype_of(tn_prec p) { return p == TN_FP64 ? 0 : 1; }

tn_status check_device_error(tn_model *m);

// Autotuner: build, capture and time (three graph replays after one warm-up,
// CUDA events on the model's stream) every candidate launch shape of a
// program, one candidate in memory at a time, and return the fastest.
// Candidates: 4 or 1 lanes x 2, 4 or 8 blocks per SM for the streaming
// absorb kernels.  Every candidate computes the same values (the shapes
// change where and in which order work runs, not any kernel's arithmetic).
tn_status autotune_program(tn_model *m, const Net &net, int kind, int dtype, int nbeta,
                           bool grads, const tn_options *opts, Tune &best) {
    double best_ms = 1e300;
    bool found = false;
    for (int lanes : {4, 1})
        for (int bps : {4, 2, 8}) {
            Tune c;
            c.max_lanes = lanes;
            c.absorb_bps = bps == 4 ? 0 : bps;
            auto C = std::make_unique<Program>();
            tn_status s = build_program(m, net, m->tree, kind, dtype, nbeta, grads, opts, *C,
                                        nullptr, &c);
            if (s == TN_E_OOM) continue;
            if (s) return s;
            s = capture_program(m, *C);
            if (s) return s;
            CK(cudaGraphLaunch(C->gexec, m->stream));
            CK(cudaEventRecord(m->ev0, m->stream));
            for (int r = 0; r < 3; ++r) CK(cudaGraphLaunch(C->gexec, m->stream));
            CK(cudaEventRecord(m->ev1, m->stream));
            CK(cudaStreamSynchronize(m->stream));
            s = check_device_error(m);
            if (s) return s;
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
                found = true;
            }
        }
    if (!found) return fail(TN_E_OOM, "no candidate program fits the device memory");
    best.tuned = true;
    return TN_OK;
}

tn_status get_program(tn_model *m, int kind, int nbeta, const tn_options *opts, bool grads,
                      Program **out) {
    tn_status s = ensure_device(m);
    if (s) return s;
    if (!m->has_tree) {
        Net net = model_net(m->md, false);
        m->tree = greedy_tree(net);
        m->has_tree = true;
    }
    tn_prec prec = opts ? opts->prec : TN_FP64;
    int dtype = dtype_of(prec);
    const bool autotune = opts && opts->autotune && (kind == K_PR || kind == K_MAR);
    auto key = std::make_tuple(kind, (int)prec, nbeta, (grads ? 1 : 0) | (autotune ? 2 : 0));
    auto it = m->progs.find(key);
    if (it != m->progs.end()) {
        *out = it->second.get();
        return TN_OK;
    }
    Net net = model_net(m->md, nbeta > 1, m->slice_vars);
    Tune tune;
    if (autotune) {
        auto tt = m->tuned.find(key);
        if (tt != m->tuned.end()) {
            tune = tt->second;
        } else {
            s = autotune_program(m, net, kind, dtype, nbeta, grads, opts, tune);
            if (s) return s;
            m->tuned[key] = tune;
        }
    }
    auto P = std::make_unique<Program>();
    s = build_program(m, net, m->tree, kind, dtype, nbeta, grads, opts, *P, nullptr, &tune);
    if (s == TN_E_OOM && !m->progs.empty()) {
        // release the other cached programs of this model and try once more
        m->progs.clear();
        P = std::make_unique<Program>();
        s = build_program(m, net, m->tree, kind, dtype, nbeta, grads, opts, *P, nullptr, &tune);
    }
    if (s) return s;
    s = capture_program(m, *P);
    if (s) return s;
    *out = P.get();
    m->progs[key] = std::move(P);
    return TN_OK;
}

tn_status check_evid(const tn_model *m, int batch, const int32_t *evid_host) {
    if (!evid_host) return TN_OK;
    for (int b = 0; b < batch; ++b)
        for (int v = 0; v < m->md.nvars; ++v) {
            int e = evid_host[(int64_t)b * m->md.nvars + v];
            if (e < -1 || e >= m->md.card[v])
                return fail(TN_E_ARG, "evidence value out of range for variable " + std::to_string(v));
        }
    return TN_OK;
}

// A bounded device-side wait that gave up leaves a flag; report and clear it.
tn_status check_device_error(tn_model *m) {
    int e = 0;
    CK(cudaMemcpy(&e, m->d_err, 4, cudaMemcpyDeviceToHost));
    if (e) {
        CK(cudaMemset(m->d_err, 0, 4));
        return fail(TN_E_TIMEOUT, "a device-side wait exceeded its time limit");
    }
    return TN_OK;
}

// Run a captured program: copy the evidence in, replay the graph, time it.
tn_status run_program(tn_model *m, Program &P, const int32_t *evid, bool evid_on_device,
                      cudaStream_t st, bool sync = true, int nrows = -1) {
    if (nrows < 0) nrows = P.nbeta;
    size_t row = (size_t)m->md.nvars * 4, eb = (size_t)P.nbeta * row;
    if (eb) {
        if (evid && nrows > 0)
            CK(cudaMemcpyAsync(P.d_evid, evid, (size_t)nrows * row,
                               evid_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        if (!evid || nrows < P.nbeta)
            CK(cudaMemsetAsync((char *)P.d_evid + (evid ? (size_t)nrows * row : 0), 0xff,
                               eb - (evid ? (size_t)nrows * row : 0), st));
    }
    if (!sync) {
        CK(cudaGraphLaunch(P.gexec, st));
        m->last_launches = P.launches;
        return TN_OK;
    }
    CK(cudaEventRecord(m->ev0, st));
    CK(cudaGraphLaunch(P.gexec, st));
    CK(cudaEventRecord(m->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->last_ms = ms;
    m->last_launches = P.launches;
    CK(cudaGetLastError());
    return check_device_error(m);
}

// Number of slice assignments and (lazily) the device table of all of them,
// last sliced variable fastest.
tn_status slice_setup(tn_model *m, int64_t &nass) {
    const auto &sl = m->slice_vars;
    nass = 1;
    for (int v : sl) nass *= m->md.card[v];
    if (sl.empty() || m->d_sl_tab) return TN_OK;
    std::vector<int32_t> tab((size_t)nass * sl.size()), var(sl.begin(), sl.end()), card;
    std::vector<int64_t> moff;
    int64_t acc = 0;
    std::vector<int64_t> off(m->md.nvars);
    for (int v = 0; v < m->md.nvars; ++v) {
        off[v] = acc;
        acc += m->md.card[v];
    }
    for (int v : sl) {
        card.push_back(m->md.card[v]);
        moff.push_back(off[v]);
    }
    for (int64_t a = 0; a < nass; ++a) {
        int64_t r = a;
        for (int j = (int)sl.size() - 1; j >= 0; --j) {
            tab[(size_t)a * sl.size() + j] = (int32_t)(r % card[j]);
            r /= card[j];
        }
    }
    CK(cudaMalloc(&m->d_sl_tab, tab.size() * 4));
    CK(cudaMemcpy(m->d_sl_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&m->d_sl_var, var.size() * 4));
    CK(cudaMemcpy(m->d_sl_var, var.data(), var.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&m->d_sl_card, card.size() * 4));
    CK(cudaMemcpy(m->d_sl_card, card.data(), card.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMalloc(&m->d_sl_moff, moff.size() * 8));
    CK(cudaMemcpy(m->d_sl_moff, moff.data(), moff.size() * 8, cudaMemcpyHostToDevice));
    return TN_OK;
}

// PR / MAR over every slice assignment: one graph replay per assignment and a
// running log-sum-exp (and Z-weighted marginals) on the device; the results
// land in the program's log Z / marginal buffers.
tn_status run_sliced(tn_model *m, Program &P, const int32_t *evid, bool evid_dev, bool marg,
                     cudaStream_t st, int nrows = -1) {
    if (nrows < 0) nrows = P.nbeta;
    int64_t nass;
    tn_status s = slice_setup(m, nass);
    if (s) return s;
    const int nsl = (int)m->slice_vars.size();
    int64_t nm = std::max<int64_t>(1, P.marg_stride);
    if (P.nbeta > m->s_cap_b || nm > m->s_cap_m) {
        for (double *p : {m->d_sM, m->d_sS, m->d_sA})
            if (p) cudaFree(p);
        m->s_cap_b = P.nbeta;
        m->s_cap_m = nm;
        CK(cudaMalloc(&m->d_sM, (size_t)P.nbeta * 8));
        CK(cudaMalloc(&m->d_sS, (size_t)P.nbeta * 8));
        CK(cudaMalloc(&m->d_sA, (size_t)P.nbeta * nm * 8));
    }
    size_t row = (size_t)m->md.nvars * 4, eb = (size_t)P.nbeta * row;
    if (eb) {
        if (evid && nrows > 0)
            CK(cudaMemcpyAsync(P.d_evid, evid, (size_t)nrows * row,
                               evid_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        if (!evid || nrows < P.nbeta)
            CK(cudaMemsetAsync((char *)P.d_evid + (evid ? (size_t)nrows * row : 0), 0xff,
                               eb - (evid ? (size_t)nrows * row : 0), st));
    }
    CK(cudaEventRecord(m->ev0, st));
    launch_slice_init(P.nbeta, nm, m->d_sM, m->d_sS, m->d_sA, st);
    for (int64_t a = 0; a < nass; ++a) {
        CK(cudaMemcpyAsync(P.d_slice_val, m->d_sl_tab + a * nsl, (size_t)nsl * 4,
                           cudaMemcpyDeviceToDevice, st));
        CK(cudaGraphLaunch(P.gexec, st));
        launch_slice_acc(P.nbeta, P.d_logz, marg ? P.d_marg : nullptr, nm, P.d_slice_val, nsl,
                         m->d_sl_var, m->d_sl_moff, m->d_sl_card, m->d_sM, m->d_sS, m->d_sA, st);
    }
    launch_slice_fin(P.nbeta, nm, m->d_sM, m->d_sS, m->d_sA, P.d_logz, marg ? P.d_marg : nullptr,
                     st);
    CK(cudaEventRecord(m->ev1, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->last_ms = ms;
    m->last_launches = (P.launches + 2) * nass + 2;
    CK(cudaGetLastError());
    return check_device_error(m);
}

cudaStream_t stream_of(tn_model *m, const tn_options *opts) {
    if (opts && opts->cuda_stream) return (cudaStream_t)opts->cuda_stream;
    return m->stream;
}

tn_status override_tables(tn_model *m, const double *dev_tables, int is_log, cudaStream_t st) {
    if (!dev_tables) {
        if (m->tables_overridden) return ensure_device(m);
        return TN_OK;
    }
    CK(cudaMemcpyAsync(m->d_tables, dev_tables, m->md.tables.size() * 8,
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(m->d_flags, is_log ? 1 : 0, 4, st));
    m->tables_overridden = true;
    return TN_OK;
}

}  // namespace

namespace tn {
// Used by other translation units of the library (declared where used).
tn_status set_error(tn_status s, const std::string &msg) { return fail(s, msg); }

// Descriptor of one plain pairwise contraction (no rescaling) on caller data.
tn_status plain_contract_desc(int nlabels, const int *sizes, int na, const int *labels_a,
                              const void *A, int nb, const int *labels_b, const void *B, int nc,
                              const int *labels_c, void *C, int semiring, int32_t *argmax,
                              CDesc &d) {
    if (nlabels < 0 || !sizes || (na && !labels_a) || (nb && !labels_b) || (nc && !labels_c) ||
        !A || !B || !C)
        return fail(TN_E_ARG, "NULL argument");
    if (semiring != 0 && semiring != 1) return fail(TN_E_ARG, "semiring must be 0 or 1");
    std::vector<int> card(sizes, sizes + nlabels);
    for (int c : card)
        if (c < 1) return fail(TN_E_ARG, "label size < 1");
    auto chk = [&](int n, const int *l, Labels &out) -> bool {
        std::set<int> seen;
        for (int i = 0; i < n; ++i) {
            if (l[i] < 0 || l[i] >= nlabels || seen.count(l[i])) return false;
            seen.insert(l[i]);
            out.push_back(l[i]);
        }
        return true;
    };
    Labels la, lb, lc;
    if (!chk(na, labels_a, la) || !chk(nb, labels_b, lb) || !chk(nc, labels_c, lc))
        return fail(TN_E_ARG, "labels out of range or repeated");
    std::set<int> u(la.begin(), la.end());
    u.insert(lb.begin(), lb.end());
    for (int v : lc)
        if (!u.count(v)) return fail(TN_E_ARG, "output label in neither operand");
    std::string err = make_desc(card, la, false, 0, A, nullptr, lb, false, 0, B, nullptr, lc,
                                false, C, nullptr, nullptr, 1, semiring == 1 ? argmax : nullptr, d);
    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
    return TN_OK;
}
}  // namespace tn

// =================================================================== C ABI

extern "C" {

const char *tn_last_error(void) { return g_err.c_str(); }

tn_status tn_load_model(const char *uai_path, tn_model **out) {
    if (!uai_path || !out) return fail(TN_E_ARG, "NULL argument");
    auto m = new (std::nothrow) tn_model();
    if (!m) return fail(TN_E_OOM, "host allocation failed");
    bool perr = false;
    std::string err = model_from_uai(uai_path, m->md, perr);
    if (!err.empty()) {
        delete m;
        return fail(perr ? TN_E_PARSE : TN_E_ARG, err);
    }
    *out = m;
    return TN_OK;
}

tn_status tn_read_evidence(const tn_model *m, const char *path, int max_sets, int32_t *evid,
                           int *nsets) {
    if (!m || !path || !nsets || max_sets < 0 || (max_sets > 0 && !evid))
        return fail(TN_E_ARG, "bad argument");
    std::vector<std::vector<int32_t>> sets;
    bool perr = false;
    std::string err = evidence_from_uai(path, m->md, sets, perr);
    if (!err.empty()) return fail(perr ? TN_E_PARSE : TN_E_ARG, err);
    *nsets = (int)sets.size();
    for (int b = 0; b < std::min<int>(max_sets, (int)sets.size()); ++b)
        std::copy(sets[b].begin(), sets[b].end(), evid + (size_t)b * m->md.nvars);
    return TN_OK;
}

tn_status tn_read_query(const tn_model *m, const char *path, int max_q, int32_t *query, int *nq) {
    if (!m || !path || !nq || max_q < 0 || (max_q > 0 && !query))
        return fail(TN_E_ARG, "bad argument");
    std::vector<int32_t> q;
    bool perr = false;
    std::string err = query_from_uai(path, m->md, q, perr);
    if (!err.empty()) return fail(perr ? TN_E_PARSE : TN_E_ARG, err);
    *nq = (int)q.size();
    std::copy(q.begin(), q.begin() + std::min<int>(max_q, (int)q.size()), query);
    return TN_OK;
}

tn_status tn_load_model_arrays(int nvars, const int *card, int nfactors, const int *scope_off,
                               const int *scope_vars, const double *tables, tn_model **out) {
    if (!out) return fail(TN_E_ARG, "NULL output");
    auto m = new (std::nothrow) tn_model();
    if (!m) return fail(TN_E_OOM, "host allocation failed");
    std::string err = model_from_arrays(nvars, card, nfactors, scope_off, scope_vars, tables, m->md);
    if (!err.empty()) {
        delete m;
        return fail(TN_E_ARG, err);
    }
    *out = m;
    return TN_OK;
}

void tn_free_model(tn_model *m) { delete m; }

tn_status tn_set_order(tn_model *m, int nnodes, const int *left, const int *right, int nslice,
                       const int *slice_vars) {
    if (!m) return fail(TN_E_ARG, "NULL model");
    int nleaves = m->md.nfactors + m->md.nvars;
    Tree t;
    t.nleaves = nleaves;
    if (nnodes == 0 && !left && !right) {
        t = greedy_tree(model_net(m->md, false));
    } else {
        if (!left || !right) return fail(TN_E_ARG, "NULL tree arrays");
        t.left.assign(left, left + nnodes);
        t.right.assign(right, right + nnodes);
        std::string err = validate_tree(t);
        if (!err.empty()) return fail(TN_E_ORDER, err);
    }
    std::vector<int> sl;
    if (nslice > 0) {
        if (!slice_vars) return fail(TN_E_ARG, "NULL slice variables");
        double nass = 1;
        for (int i = 0; i < nslice; ++i) {
            int v = slice_vars[i];
            if (v < 0 || v >= m->md.nvars) return fail(TN_E_ARG, "slice variable out of range");
            if (std::find(sl.begin(), sl.end(), v) != sl.end())
                return fail(TN_E_ARG, "slice variable repeated");
            sl.push_back(v);
            nass *= m->md.card[v];
        }
        if (nass > (double)(1 << 24)) return fail(TN_E_ARG, "more than 2^24 slices");
    }
    m->tree = t;
    m->has_tree = true;
    if (sl != m->slice_vars) {
        for (void *p : {(void *)m->d_sl_var, (void *)m->d_sl_card, (void *)m->d_sl_tab,
                        (void *)m->d_sl_moff})
            if (p) cudaFree(p);
        m->d_sl_var = m->d_sl_card = m->d_sl_tab = nullptr;
        m->d_sl_moff = nullptr;
    }
    m->slice_vars = sl;
    m->progs.clear();
    return TN_OK;
}

tn_status tn_tree_from_elimination(const tn_model *m, int nelim, const int *order, int *left,
                                   int *right) {
    if (!m || (!order && nelim) || !left || !right) return fail(TN_E_ARG, "NULL argument");
    std::vector<int> o(order, order + nelim);
    for (int v : o)
        if (v < 0 || v >= m->md.nvars) return fail(TN_E_ARG, "order variable out of range");
    Tree t = tree_from_elimination(model_net(m->md, false), o);
    std::copy(t.left.begin(), t.left.end(), left);
    std::copy(t.right.begin(), t.right.end(), right);
    return TN_OK;
}

tn_status tn_optimize_order(const tn_model *m, int method, int restarts, uint64_t seed, int *left,
                            int *right) {
    if (!m || !left || !right) return fail(TN_E_ARG, "NULL argument");
    if (method < 0 || method > 4) return fail(TN_E_ARG, "unknown method");
    Tree t = optimize_tree(model_net(m->md, false), method, restarts, seed);
    std::copy(t.left.begin(), t.left.end(), left);
    std::copy(t.right.begin(), t.right.end(), right);
    return TN_OK;
}

tn_status tn_choose_slices(const tn_model *m, const int *left, const int *right,
                           double target_sc_log2, int max_vars, int *vars, int *nvars_out) {
    if (!m || !vars || !nvars_out || max_vars < 0) return fail(TN_E_ARG, "bad argument");
    Tree t;
    if (left && right) {
        t.nleaves = (int)model_net(m->md, false).leaf.size();
        t.left.assign(left, left + t.nleaves - 1);
        t.right.assign(right, right + t.nleaves - 1);
        std::string err = validate_tree(t);
        if (!err.empty()) return fail(TN_E_ORDER, err);
    } else {
        t = m->has_tree ? m->tree : greedy_tree(model_net(m->md, false));
    }
    // sc (log2 entries of the largest intermediate), tc (log2 multiply-adds
    // over all slices) and the largest node of the tree with `sl` sliced
    auto cost = [&](const std::vector<int> &sl, double &sc, double &tc, int &big) {
        Plan p;
        build_plan(model_net(m->md, false, sl), t, p);
        double nass = 1;
        for (int v : sl) nass *= m->md.card[v];
        sc = 0;
        tc = 0;
        big = -1;
        const int n = t.nleaves;
        for (int id = n; id < 2 * n - 1; ++id) {
            double e = std::log2((double)p.node[id].size);
            if (e > sc) {
                sc = e;
                big = id;
            }
            tc += p.node[id].muladds;
        }
        tc = std::log2(std::max(1.0, tc * nass));
        return p;
    };
    std::vector<int> sl;
    double sc, tc;
    int big;
    Plan p = cost(sl, sc, tc, big);
    while ((int)sl.size() < max_vars && sc > target_sc_log2 && big >= 0) {
        // candidates: the labels of the current largest intermediate
        Labels cand = p.node[big].labels;
        int bestv = -1;
        double bsc = 0, btc = 0;
        for (int v : cand) {
            std::vector<int> trial = sl;
            trial.push_back(v);
            double s2, t2;
            int b2;
            cost(trial, s2, t2, b2);
            if (bestv < 0 || s2 < bsc || (s2 == bsc && t2 < btc)) {
                bestv = v;
                bsc = s2;
                btc = t2;
            }
        }
        if (bestv < 0) break;
        sl.push_back(bestv);
        p = cost(sl, sc, tc, big);
    }
    std::copy(sl.begin(), sl.end(), vars);
    *nvars_out = (int)sl.size();
    return TN_OK;
}

tn_status tn_reassociate(const tn_model *m, const int *left, const int *right, int *left_out,
                         int *right_out) {
    if (!m || !left || !right || !left_out || !right_out) return fail(TN_E_ARG, "NULL argument");
    Net net = model_net(m->md, false);
    Tree t;
    t.nleaves = (int)net.leaf.size();
    t.left.assign(left, left + t.nleaves - 1);
    t.right.assign(right, right + t.nleaves - 1);
    std::string err = validate_tree(t);
    if (!err.empty()) return fail(TN_E_ORDER, err);
    Tree r = reassociate_chains(net, t);
    std::copy(r.left.begin(), r.left.end(), left_out);
    std::copy(r.right.begin(), r.right.end(), right_out);
    return TN_OK;
}

tn_status tn_tree_stats(const tn_model *m, int batch, tn_prec prec, double *out) {
    if (!m || !out || batch < 1) return fail(TN_E_ARG, "bad argument");
    Net net = model_net(m->md, batch > 1, m->slice_vars);
    Tree t = m->has_tree ? m->tree : greedy_tree(model_net(m->md, false));
    Plan p;
    std::string err = build_plan(net, t, p);
    double nass = 1;
    for (int v : m->slice_vars) nass *= m->md.card[v];
    if (!err.empty()) return fail(TN_E_ORDER, err);
    int n = t.nleaves;
    double mul = 0, bytes = 0, sc = 0;
    double es = prec == TN_FP64 ? 8 : 4;
    for (int id = n; id < 2 * n - 1; ++id) {
        const Node &nd = p.node[id];
        double bt = nd.beta ? batch : 1;
        mul += nd.muladds * bt;
        bytes += es * ((double)p.node[nd.a].size * (p.node[nd.a].beta ? batch : 1) +
                       (double)p.node[nd.b].size * (p.node[nd.b].beta ? batch : 1) +
                       (double)nd.size * bt);
        sc = std::max(sc, std::log2((double)nd.size * bt));
    }
    mul *= nass;
    bytes *= nass;
    out[0] = mul > 0 ? std::log2(mul) : 0;
    out[1] = sc;
    out[2] = bytes > 0 ? std::log2(bytes / es) : 0;
    out[3] = n - 1;
    out[4] = 2 * mul;
    out[5] = bytes;
    return TN_OK;
}

// The program for `batch` evidence sets, or, when it does not fit the device
// memory / HBM budget, for the largest power-of-two sub-batch that does.
static tn_status program_fitting(tn_model *m, int kind, int batch, const tn_options *opts,
                                 bool grads, Program **out, int *sub) {
    int b = batch;
    for (;;) {
        tn_status s = get_program(m, kind, b, opts, grads, out);
        if (s == TN_OK) {
            *sub = b;
            return TN_OK;
        }
        if (s != TN_E_OOM || b == 1) return s;
        int p = 1;
        while (p * 2 < b) p *= 2;
        b = p;
    }
}

static tn_status pr_common(tn_model *m, int batch, const int32_t *evid, bool evid_dev,
                           const double *tables_dev, int is_log, const tn_options *opts,
                           double *logz, bool logz_dev) {
    if (!m || batch < 1 || !logz) return fail(TN_E_ARG, "bad argument");
    if (!evid_dev) {
        tn_status s = check_evid(m, batch, evid);
        if (s) return s;
    }
    Program *P;
    int sub = batch;
    tn_status s = program_fitting(m, K_PR, batch, opts, false, &P, &sub);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, tables_dev, is_log, st);
    if (s) return s;
    const bool async =
        evid_dev && opts && opts->cuda_stream && m->slice_vars.empty() && sub == batch;
    double ms = 0;
    for (int i = 0; i < batch; i += sub) {
        int nr = std::min(sub, batch - i);
        const int32_t *ev = evid ? evid + (size_t)i * m->md.nvars : nullptr;
        s = m->slice_vars.empty() ? run_program(m, *P, ev, evid_dev, st, !async, nr)
                                  : run_sliced(m, *P, ev, evid_dev, false, st, nr);
        if (s) return s;
        ms += m->last_ms;
        CK(cudaMemcpyAsync(logz + i, P->d_logz, (size_t)nr * 8,
                           logz_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    if (!async) {
        CK(cudaStreamSynchronize(st));
        m->last_ms = ms;
    }
    return TN_OK;
}

tn_status tn_pr(tn_model *m, int batch, const int32_t *evid, const tn_options *opts, double *logz) {
    return pr_common(m, batch, evid, false, nullptr, 0, opts, logz, false);
}

tn_status tn_pr_dev(tn_model *m, int batch, const int32_t *evid, const double *factor_tables,
                    int tables_are_log, const tn_options *opts, double *logz) {
    return pr_common(m, batch, evid, true, factor_tables, tables_are_log, opts, logz, true);
}

static tn_status mar_common(tn_model *m, int batch, const int32_t *evid, bool dev,
                            const double *tables_dev, int is_log, const tn_options *opts,
                            double *logz, double *marg, double *grad) {
    if (!m || batch < 1 || !logz || !marg) return fail(TN_E_ARG, "bad argument");
    if (!dev) {
        tn_status s = check_evid(m, batch, evid);
        if (s) return s;
    }
    Program *P;
    int sub = batch;
    tn_status s = program_fitting(m, K_MAR, batch, opts, grad != nullptr, &P, &sub);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, tables_dev, is_log, st);
    if (s) return s;
    const bool async = dev && opts && opts->cuda_stream && m->slice_vars.empty() && sub == batch;
    cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double ms = 0;
    for (int i = 0; i < batch; i += sub) {
        int nr = std::min(sub, batch - i);
        const int32_t *ev = evid ? evid + (size_t)i * m->md.nvars : nullptr;
        s = m->slice_vars.empty() ? run_program(m, *P, ev, dev, st, !async, nr)
                                  : run_sliced(m, *P, ev, dev, true, st, nr);
        if (s) return s;
        ms += m->last_ms;
        CK(cudaMemcpyAsync(logz + i, P->d_logz, (size_t)nr * 8, k, st));
        CK(cudaMemcpyAsync(marg + (size_t)i * P->marg_stride, P->d_marg,
                           (size_t)nr * P->marg_stride * 8, k, st));
        if (grad)
            CK(cudaMemcpyAsync(grad + (size_t)i * P->grad_stride, P->d_grad,
                               (size_t)nr * P->grad_stride * 8, k, st));
    }
    if (async) return TN_OK;
    CK(cudaStreamSynchronize(st));
    m->last_ms = ms;
    if (!dev) {
        for (int b = 0; b < batch; ++b)
            if (!(logz[b] > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0 for evidence set " + std::to_string(b));
    }
    return TN_OK;
}

tn_status tn_mar(tn_model *m, int batch, const int32_t *evid, const tn_options *opts, double *logz,
                 double *marg) {
    return mar_common(m, batch, evid, false, nullptr, 0, opts, logz, marg, nullptr);
}

// Several models in one launch: each model's captured program becomes a
// child graph of one parent graph (independent branches, so the device runs
// them concurrently: a model of small treewidth no longer pays a launch and
// an idle GPU of its own), launched once on one stream.
tn_status tn_solve_multi(int task, int nmodels, tn_model *const *models, const int *batch,
                         const int32_t *const *evid, const tn_options *opts,
                         double *const *logz, double *const *marg) {
    if (nmodels < 1 || !models || !batch || !logz || (task != 0 && task != 1) ||
        (task == 1 && !marg))
        return fail(TN_E_ARG, "bad argument");
    std::vector<Program *> progs(nmodels);
    int dev = -1;
    for (int i = 0; i < nmodels; ++i) {
        tn_model *m = models[i];
        if (!m || batch[i] < 1 || !logz[i] || (task == 1 && !marg[i]))
            return fail(TN_E_ARG, "bad argument for model " + std::to_string(i));
        for (int j = 0; j < i; ++j)
            if (models[j] == m) return fail(TN_E_ARG, "a model appears twice");
        if (!m->slice_vars.empty()) return fail(TN_E_UNSUPPORTED, "sliced model in a multi-model launch");
        tn_status s = check_evid(m, batch[i], evid ? evid[i] : nullptr);
        if (s) return s;
        s = get_program(m, task == 0 ? K_PR : K_MAR, batch[i], opts, false, &progs[i]);
        if (s) return s;
        if (dev < 0) dev = m->device;
        else if (m->device != dev) return fail(TN_E_ARG, "models on different devices");
        s = override_tables(m, nullptr, 0, m->stream);
        if (s) return s;
    }
    cudaStream_t st = opts && opts->cuda_stream ? (cudaStream_t)opts->cuda_stream : models[0]->stream;
    for (int i = 0; i < nmodels; ++i) CK(cudaStreamSynchronize(models[i]->stream));
    cudaGraph_t parent = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaGraphCreate(&parent, 0));
    tn_status rs = TN_OK;
    for (int i = 0; i < nmodels && rs == TN_OK; ++i) {
        cudaGraphNode_t node;
        cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, progs[i]->graph);
        if (e != cudaSuccess) rs = fail(TN_E_CUDA, std::string("child graph: ") + cudaGetErrorString(e));
    }
    if (rs == TN_OK) {
        cudaError_t e = cudaGraphInstantiate(&exec, parent, 0);
        if (e != cudaSuccess) rs = fail(TN_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    if (rs == TN_OK) {
        for (int i = 0; i < nmodels; ++i) {
            Program *P = progs[i];
            size_t eb = (size_t)P->nbeta * models[i]->md.nvars * 4;
            if (!eb) continue;
            if (evid && evid[i])
                CK(cudaMemcpyAsync(P->d_evid, evid[i], eb, cudaMemcpyHostToDevice, st));
            else
                CK(cudaMemsetAsync(P->d_evid, 0xff, eb, st));
        }
        CK(cudaEventRecord(models[0]->ev0, st));
        CK(cudaGraphLaunch(exec, st));
        CK(cudaEventRecord(models[0]->ev1, st));
        for (int i = 0; i < nmodels; ++i) {
            Program *P = progs[i];
            CK(cudaMemcpyAsync(logz[i], P->d_logz, (size_t)batch[i] * 8, cudaMemcpyDeviceToHost, st));
            if (task == 1)
                CK(cudaMemcpyAsync(marg[i], P->d_marg, (size_t)batch[i] * P->marg_stride * 8,
                                   cudaMemcpyDeviceToHost, st));
        }
        CK(cudaStreamSynchronize(st));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, models[0]->ev0, models[0]->ev1));
        int64_t nl = 0;
        for (int i = 0; i < nmodels; ++i) nl += progs[i]->launches;
        for (int i = 0; i < nmodels && rs == TN_OK; ++i) {
            models[i]->last_ms = ms;
            models[i]->last_launches = nl;
            rs = check_device_error(models[i]);
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(parent);
    if (rs) return rs;
    if (task == 1)
        for (int i = 0; i < nmodels; ++i)
            for (int b = 0; b < batch[i]; ++b)
                if (!(logz[i][b] > -INFINITY))
                    return fail(TN_E_ARG, "p(e) = 0 for evidence set " + std::to_string(b) +
                                              " of model " + std::to_string(i));
    return TN_OK;
}

tn_status tn_mar_dev(tn_model *m, int batch, const int32_t *evid, const double *factor_tables,
                     int tables_are_log, const tn_options *opts, double *logz, double *marg,
                     double *grad) {
    return mar_common(m, batch, evid, true, factor_tables, tables_are_log, opts, logz, marg,
                      grad);
}

// Joint marginal of a variable set Q: p(Q = q, e) is the contraction with Q
// left open (Eq. evidence); with Q's labels sliced, each slice is the PR of
// the evidence extended by Q = q (Eq. pr), so the slices run as the rows of
// one batched PR along the model's tree.  Rows whose assignment contradicts
// an observed query variable are not run (their probability is 0).
static constexpr int64_t kJointMaxRows = 1 << 16;

tn_status tn_joint_mar(tn_model *m, const int32_t *evid, int nq, const int32_t *query,
                       const tn_options *opts, double *logz, double *joint) {
    if (!m || nq < 1 || !query || !logz || !joint) return fail(TN_E_ARG, "bad argument");
    const int nv = m->md.nvars;
    if (nq > nv) return fail(TN_E_ARG, "more query variables than variables");
    tn_status s = check_evid(m, 1, evid);
    if (s) return s;
    std::vector<char> seen(nv, 0);
    int64_t rows = 1;
    for (int i = 0; i < nq; ++i) {
        const int v = query[i];
        if (v < 0 || v >= nv) return fail(TN_E_ARG, "query variable out of range");
        if (seen[v]) return fail(TN_E_ARG, "query variable " + std::to_string(v) + " repeated");
        seen[v] = 1;
        rows *= m->md.card[v];
        if (rows > kJointMaxRows)
            return fail(TN_E_ARG, "joint domain of the query holds more than 65536 assignments");
    }
    std::vector<int32_t> ev;
    std::vector<int64_t> at;   // joint index of each batch row
    std::vector<int32_t> row(nv);
    for (int64_t r = 0; r < rows; ++r) {
        for (int v = 0; v < nv; ++v) row[v] = evid ? evid[v] : -1;
        bool ok = true;
        int64_t x = r;
        for (int i = nq - 1; i >= 0; --i) {   // the last query variable varies fastest
            const int v = query[i], c = m->md.card[v];
            const int32_t a = (int32_t)(x % c);
            x /= c;
            if (row[v] >= 0 && row[v] != a) ok = false;
            row[v] = a;
        }
        if (!ok) continue;
        ev.insert(ev.end(), row.begin(), row.end());
        at.push_back(r);
    }
    std::fill(joint, joint + rows, 0.0);
    std::vector<double> lz(at.size());
    s = tn_pr(m, (int)at.size(), ev.data(), opts, lz.data());
    if (s) return s;
    // log p(e) = log sum_q p(Q = q, e)
    double mx = -INFINITY;
    for (double v : lz) mx = std::max(mx, v);
    if (!(mx > -INFINITY)) {
        *logz = -INFINITY;
        return fail(TN_E_ARG, "p(e) = 0");
    }
    double sum = 0;
    for (double v : lz) sum += std::exp(v - mx);
    *logz = mx + std::log(sum);
    for (size_t k = 0; k < at.size(); ++k) joint[at[k]] = std::exp(lz[k] - *logz);
    return TN_OK;
}

tn_status tn_map(tn_model *m, const int32_t *evid, const tn_options *opts, int32_t *assign,
                 double *logp) {
    if (!m || !assign || !logp) return fail(TN_E_ARG, "bad argument");
    if (!m->slice_vars.empty())
        return fail(TN_E_UNSUPPORTED, "this task does not run on a sliced tree; set the order without slices");
    tn_status s = check_evid(m, 1, evid);
    if (s) return s;
    Program *P;
    s = get_program(m, K_MAP, 1, opts, false, &P);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, nullptr, 0, st);
    if (s) return s;
    s = run_program(m, *P, evid, false, st);
    if (s) return s;
    CK(cudaMemcpyAsync(logp, P->d_logz, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(assign, P->d_assign, (size_t)m->md.nvars * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!(*logp > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
    return TN_OK;
}

// Draw n samples into d_out from the program's cached forward tensors (the
// last run), with the Philox key `seed`.
static tn_status draw_samples(tn_model *m, Program &P, int64_t n, uint64_t seed, int8_t *d_out,
                              cudaStream_t st) {
    if (n == 0) return TN_OK;
    int64_t coff = 0;
    for (auto &c : P.cdf_nodes) {
        // cumulative tables of the nodes with large summed spaces
        if (P.dtype == 0) launch_cdf_rows<double>(c.first, c.second, P.cdf + coff, st);
        else launch_cdf_rows<float>(c.first, c.second, P.cdf + coff, st);
        coff += c.second * c.first.ktotal;
    }
    if (P.dtype == 0)
        launch_sample<double>(P.d_meta, P.nmeta, (const double *)P.arena, P.cdf, P.d_evid,
                              m->md.nvars, n, seed, d_out, st);
    else
        launch_sample<float>(P.d_meta, P.nmeta, (const float *)P.arena, P.cdf, P.d_evid,
                             m->md.nvars, n, seed, d_out, st);
    CK(cudaGetLastError());
    return TN_OK;
}

static uint64_t mix64(uint64_t x) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014)
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

tn_status tn_sample(tn_model *m, const int32_t *evid, uint64_t seed, int64_t n,
                    const tn_options *opts, int8_t *samples) {
    if (!m || n < 0 || (!samples && n)) return fail(TN_E_ARG, "bad argument");
    for (int v = 0; v < m->md.nvars; ++v)
        if (m->md.card[v] > 127) return fail(TN_E_UNSUPPORTED, "domain size above 127");
    tn_status s = check_evid(m, 1, evid);
    if (s) return s;
    Program *P;
    s = get_program(m, K_SAMPLE, 1, opts, false, &P);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, nullptr, 0, st);
    if (s) return s;
    const int nv = m->md.nvars;
    if (m->slice_vars.empty()) {
        s = run_program(m, *P, evid, false, st);
        if (s) return s;
        double lz;
        CK(cudaMemcpy(&lz, P->d_logz, 8, cudaMemcpyDeviceToHost));
        if (!(lz > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
        if (n == 0) return TN_OK;
        int8_t *d_out = nullptr;
        CK(cudaMallocAsync(&d_out, (size_t)n * nv, st));
        CK(cudaEventRecord(m->ev0, st));
        s = draw_samples(m, *P, n, seed, d_out, st);
        if (s) return s;
        CK(cudaEventRecord(m->ev1, st));
        CK(cudaMemcpyAsync(samples, d_out, (size_t)n * nv, cudaMemcpyDeviceToHost, st));
        CK(cudaFreeAsync(d_out, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
        m->last_ms += ms;
        CK(cudaGetLastError());
        return TN_OK;
    }
    // Sliced tree: p(x) = sum_a p(a) p(x | a) with p(a) = Z_a / Z over the
    // assignments a of the sliced variables.  Pass 1 computes every Z_a, the
    // number of samples per assignment is drawn from the multinomial, pass 2
    // re-runs each drawn assignment's forward pass (its tensors are the
    // cache) and samples within it; the rows are shuffled at the end.
    int64_t nass;
    s = slice_setup(m, nass);
    if (s) return s;
    const int nsl = (int)m->slice_vars.size();
    std::vector<int32_t> ev(nv, -1);
    if (evid) std::copy(evid, evid + nv, ev.begin());
    double tms = 0;
    // forward pass of assignment a; `possible` false when the evidence rules it out
    auto run_assignment = [&](int64_t a, bool &possible) -> tn_status {
        std::vector<int32_t> ea = ev;
        int64_t r = a;
        possible = true;
        for (int j = nsl - 1; j >= 0; --j) {
            const int v = m->slice_vars[j], c = m->md.card[v];
            const int32_t val = (int32_t)(r % c);
            r /= c;
            if (ea[v] >= 0 && ea[v] != val) possible = false;
            ea[v] = val;
        }
        if (!possible) return TN_OK;
        CK(cudaMemcpyAsync(P->d_slice_val, m->d_sl_tab + a * nsl, (size_t)nsl * 4,
                           cudaMemcpyDeviceToDevice, st));
        tn_status e = run_program(m, *P, ea.data(), false, st);
        tms += m->last_ms;
        return e;
    };
    std::vector<double> lz(nass, -INFINITY);
    for (int64_t a = 0; a < nass; ++a) {
        bool ok;
        s = run_assignment(a, ok);
        if (s) return s;
        if (!ok) continue;
        CK(cudaMemcpy(&lz[a], P->d_logz, 8, cudaMemcpyDeviceToHost));
        if (!(lz[a] > -INFINITY)) lz[a] = -INFINITY;
    }
    double mx = -INFINITY;
    for (double v : lz) mx = std::max(mx, v);
    if (!(mx > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
    std::vector<double> cum(nass);
    double acc = 0;
    for (int64_t a = 0; a < nass; ++a) {
        acc += lz[a] > -INFINITY ? std::exp(lz[a] - mx) : 0.0;
        cum[a] = acc;
    }
    if (n == 0) return TN_OK;
    std::mt19937_64 rng(mix64(seed ^ 0x5ca1ab1eull));
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::vector<int64_t> cnt(nass, 0);
    for (int64_t i = 0; i < n; ++i) {
        const double u = U(rng) * acc;
        int64_t a = std::upper_bound(cum.begin(), cum.end(), u) - cum.begin();
        cnt[std::min(a, nass - 1)]++;
    }
    int8_t *d_out = nullptr;
    CK(cudaMallocAsync(&d_out, (size_t)n * nv, st));
    int64_t off = 0;
    for (int64_t a = 0; a < nass; ++a) {
        if (!cnt[a]) continue;
        bool ok;
        s = run_assignment(a, ok);
        if (s) return s;
        CK(cudaEventRecord(m->ev0, st));
        s = draw_samples(m, *P, cnt[a], mix64(seed + (uint64_t)a), d_out + off * nv, st);
        if (s) return s;
        CK(cudaEventRecord(m->ev1, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
        tms += ms;
        off += cnt[a];
    }
    std::vector<int8_t> h((size_t)n * nv);
    CK(cudaMemcpyAsync(h.data(), d_out, h.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(d_out, st));
    CK(cudaStreamSynchronize(st));
    // rows grouped by assignment -> a uniformly random order (Fisher-Yates)
    std::vector<int64_t> perm(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = std::min(i, (int64_t)(U(rng) * (double)(i + 1)));
        std::swap(perm[i], perm[j]);
    }
    for (int64_t i = 0; i < n; ++i)
        std::copy(h.begin() + perm[i] * nv, h.begin() + (perm[i] + 1) * nv, samples + i * nv);
    m->last_ms = tms;
    CK(cudaGetLastError());
    return check_device_error(m);
}

// MMAP by the two-phase method of Sec. MMAP: (1) partition the factors so
// that every summed variable (neither queried nor observed) has all of its
// factors in one group -- union of factors sharing a summed variable;
// (2) sum-contract each group to a tensor over its query variables;
// (3) solve MPE over the query variables on the network of those tensors, the
// factors that hold no summed variable, and the query unity vectors.
// Evidence enters every network that holds an observed variable as that
// variable's indicator vector (the indicator is idempotent, so copies in
// several networks slice each factor exactly once).
tn_status tn_mmap(tn_model *m, const int32_t *evid, int nq, const int32_t *query,
                  const tn_options *opts, int32_t *assign, double *logp) {
    if (!m || nq < 1 || !query || !assign || !logp) return fail(TN_E_ARG, "bad argument");
    tn_status s = check_evid(m, 1, evid);
    if (s) return s;
    const ModelData &md = m->md;
    std::vector<char> isq(md.nvars, 0), ise(md.nvars, 0);
    for (int i = 0; i < nq; ++i) {
        int q = query[i];
        if (q < 0 || q >= md.nvars) return fail(TN_E_ARG, "query variable out of range");
        if (isq[q]) return fail(TN_E_ARG, "query variable repeated");
        isq[q] = 1;
    }
    for (int v = 0; v < md.nvars; ++v) {
        ise[v] = evid && evid[v] >= 0;
        if (ise[v] && isq[v]) return fail(TN_E_ARG, "query overlaps the evidence");
    }
    s = ensure_device(m);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, nullptr, 0, st);
    if (s) return s;
    tn_prec prec = opts ? opts->prec : TN_FP64;
    int dtype = dtype_of(prec);
    std::vector<int8_t> key(md.nvars + 1);
    for (int v = 0; v < md.nvars; ++v) key[v] = isq[v] ? 1 : ise[v] ? 2 : 0;
    key[md.nvars] = (int8_t)(dtype * 4 + (int)prec);
    // results of the top-level MPE program: log p and the assignment
    auto finish = [&](Program &P2, double lconst, double ms, int64_t launches) -> tn_status {
        double lp;
        std::vector<int32_t> x(md.nvars);
        CK(cudaMemcpyAsync(&lp, P2.d_logz, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(x.data(), P2.d_assign, (size_t)md.nvars * 4, cudaMemcpyDeviceToHost,
                           st));
        CK(cudaStreamSynchronize(st));
        *logp = lp + lconst;
        for (int i = 0; i < nq; ++i) assign[i] = x[query[i]];
        m->last_launches = launches;
        m->last_ms = ms;
        if (!(lp > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
        return TN_OK;
    };
    if (m->mmap && m->mmap->key == key) {
        double ms = 0;
        int64_t launches = 0;
        for (auto &P : m->mmap->groups) {
            s = run_program(m, *P, evid, false, st);
            if (s) return s;
            ms += m->last_ms;
            launches += P->launches;
        }
        s = run_program(m, *m->mmap->top, evid, false, st);
        if (s) return s;
        return finish(*m->mmap->top, m->mmap->lconst, ms + m->last_ms,
                      launches + m->mmap->top->launches);
    }
    m->mmap.reset();
    double build_ms = 0;
    // union-find over factors sharing a summed variable
    std::vector<int> par(md.nfactors);
    std::iota(par.begin(), par.end(), 0);
    auto find = [&](int x) {
        while (par[x] != x) x = par[x] = par[par[x]];
        return x;
    };
    std::vector<int> first(md.nvars, -1);
    for (int f = 0; f < md.nfactors; ++f)
        for (int v : md.scope[f]) {
            if (isq[v] || ise[v]) continue;
            if (first[v] < 0) first[v] = f;
            else par[find(f)] = find(first[v]);
        }
    std::map<int, std::vector<int>> groups;
    std::vector<int> ungrouped;
    for (int f = 0; f < md.nfactors; ++f) {
        bool has_summed = false;
        for (int v : md.scope[f]) has_summed |= !isq[v] && !ise[v];
        if (has_summed) groups[find(f)].push_back(f);
        else ungrouped.push_back(f);
    }
    double lconst = 0;   // summed variables that occur in no factor
    {
        std::vector<char> seen(md.nvars, 0);
        for (int f = 0; f < md.nfactors; ++f)
            for (int v : md.scope[f]) seen[v] = 1;
        for (int v = 0; v < md.nvars; ++v)
            if (!seen[v] && !isq[v] && !ise[v]) lconst += std::log((double)md.card[v]);
    }
    std::vector<std::unique_ptr<Program>> progs;
    Net net2;
    net2.card = md.card;
    std::vector<LeafRec> spec2;
    int64_t launches = 0;
    for (auto &g : groups) {
        Net net;
        net.card = md.card;
        std::vector<LeafRec> spec;
        std::set<int> vars;
        for (int f : g.second) {
            net.leaf.push_back(md.scope[f]);
            net.leaf_beta.push_back(0);
            LeafRec r;
            std::memset(&r, 0, sizeof r);
            r.kind = LEAF_FACTOR;
            r.src = md.toff[f];
            spec.push_back(r);
            for (int v : md.scope[f]) vars.insert(v);
        }
        for (int v : vars) {
            if (isq[v]) {
                net.out.push_back(v);
                continue;
            }
            net.leaf.push_back({v});
            net.leaf_beta.push_back(0);
            LeafRec r;
            std::memset(&r, 0, sizeof r);
            r.kind = LEAF_UNITY;
            r.var = v;
            spec.push_back(r);
        }
        Tree t = optimize_tree(net, 1, 4, 12345);
        auto P = std::make_unique<Program>();
        s = build_program(m, net, t, K_SUMNET, dtype, 1, false, opts, *P, &spec);
        if (s) return s;
        s = capture_program(m, *P);
        if (s) return s;
        s = run_program(m, *P, evid, false, st);
        if (s) return s;
        build_ms += m->last_ms;
        launches += P->launches;
        const Node &root = P->plan.node[P->plan.root];
        net2.leaf.push_back(root.labels);
        net2.leaf_beta.push_back(0);
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        r.kind = LEAF_EXTERNAL;
        r.src = (int64_t)(uintptr_t)(P->arena + P->fwd[P->plan.root].off * P->esz);
        r.sigma = P->d_sigma;
        r.size = root.size;
        spec2.push_back(r);
        progs.push_back(std::move(P));
    }
    std::set<int> evars2;
    for (int f : ungrouped) {
        net2.leaf.push_back(md.scope[f]);
        net2.leaf_beta.push_back(0);
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        r.kind = LEAF_FACTOR;
        r.src = md.toff[f];
        spec2.push_back(r);
        for (int v : md.scope[f])
            if (ise[v]) evars2.insert(v);
    }
    std::vector<int> qs(query, query + nq);
    std::sort(qs.begin(), qs.end());
    for (int v : qs) evars2.insert(v);
    for (int v : evars2) {
        net2.leaf.push_back({v});
        net2.leaf_beta.push_back(0);
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        r.kind = LEAF_UNITY;
        r.var = v;
        spec2.push_back(r);
    }
    if (net2.leaf.size() < 2) {
        net2.leaf.push_back({});
        net2.leaf_beta.push_back(0);
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        r.kind = LEAF_EXTERNAL;
        spec2.push_back(r);
        return fail(TN_E_UNSUPPORTED, "MMAP network with a single tensor");
    }
    Tree t2 = optimize_tree(net2, 1, 4, 54321);
    auto P2 = std::make_unique<Program>();
    s = build_program(m, net2, t2, K_MAP, dtype, 1, false, opts, *P2, &spec2);
    if (s) return s;
    s = capture_program(m, *P2);
    if (s) return s;
    s = run_program(m, *P2, evid, false, st);
    if (s) return s;
    build_ms += m->last_ms;
    launches += P2->launches;
    auto c = std::make_unique<MmapCache>();
    c->key = key;
    c->groups = std::move(progs);
    c->top = std::move(P2);
    c->lconst = lconst;
    m->mmap = std::move(c);
    return finish(*m->mmap->top, lconst, build_ms, launches);
}

// One pairwise contraction on caller-provided device buffers.
// One wait-timeout flag per device for the single-contraction entry points,
// created on first use.
static tn_status device_err_flag(int **out) {
    static std::mutex err_mu;
    static std::map<int, int *> err_flags;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(err_mu);
    int *&f = err_flags[dev];
    if (!f) {
        CK(cudaMalloc(&f, 16));
        CK(cudaMemset(f, 0, 16));
    }
    *out = f;
    return TN_OK;
}

tn_status tn_contract_dev(int nlabels, const int *sizes, int na, const int *labels_a,
                          const void *A, int nb, const int *labels_b, const void *B, int nc,
                          const int *labels_c, void *C, int semiring, int dtype, tn_prec prec,
                          int32_t *argmax, void *cuda_stream) {
    if (nlabels < 0 || !sizes || (na && !labels_a) || (nb && !labels_b) || (nc && !labels_c) ||
        !A || !B || !C)
        return fail(TN_E_ARG, "NULL argument");
    if (semiring != 0 && semiring != 1) return fail(TN_E_ARG, "semiring must be 0 or 1");
    if (dtype != 0 && dtype != 1) return fail(TN_E_ARG, "dtype must be 0 or 1");
    std::vector<int> card(sizes, sizes + nlabels);
    for (int c : card)
        if (c < 1) return fail(TN_E_ARG, "label size < 1");
    auto chk = [&](int n, const int *l, Labels &out) -> bool {
        std::set<int> seen;
        for (int i = 0; i < n; ++i) {
            if (l[i] < 0 || l[i] >= nlabels || seen.count(l[i])) return false;
            seen.insert(l[i]);
            out.push_back(l[i]);
        }
        return true;
    };
    Labels la, lb, lc;
    if (!chk(na, labels_a, la) || !chk(nb, labels_b, lb) || !chk(nc, labels_c, lc))
        return fail(TN_E_ARG, "labels out of range or repeated");
    {
        std::set<int> u(la.begin(), la.end());
        u.insert(lb.begin(), lb.end());
        for (int v : lc)
            if (!u.count(v)) return fail(TN_E_ARG, "output label in neither operand");
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // GEMM form for dense sum-product contractions (every group >= 64 entries)
    if (semiring == 0) {
        std::set<int> sa(la.begin(), la.end()), sb(lb.begin(), lb.end()), sc(lc.begin(), lc.end());
        Labels bt, gm, gn, gk;
        bool onesided = false;
        for (int v : la) {
            if (sc.count(v)) (sb.count(v) ? bt : gm).push_back(v);
            else if (sb.count(v)) gk.push_back(v);
            else onesided = true;
        }
        for (int v : lb)
            if (sc.count(v) && !sa.count(v)) gn.push_back(v);
            else if (!sc.count(v) && !sa.count(v)) onesided = true;
        auto prod = [&](const Labels &l) {
            int64_t q = 1;
            for (int v : l) q *= card[v];
            return q;
        };
        if (!onesided && prod(gm) >= 64 && prod(gn) >= 64 && prod(gk) >= 64) {
            int store_t = dtype == 0 ? E_F64 : E_F32;
            int gemm_t = dtype == 0 ? E_F64 : prec == TN_BF16 ? E_BF16 : E_F32;
            Opnd X{&la, false, 0, A, nullptr}, Y{&lb, false, 0, B, nullptr};
            GemmOp op;
            size_t nx, ny, nd;
            std::string e = make_gemm_op(card, 1, store_t, gemm_t, X, Y, bt, gm, gn, gk, lc, false,
                                         C, nullptr, op, nx, ny, nd);
            if (!e.empty()) return fail(TN_E_UNSUPPORTED, e);
            void *wx = nullptr, *wy = nullptr, *wd = nullptr;
            CK(cudaMallocAsync(&wx, nx, st));
            CK(cudaMallocAsync(&wy, ny, st));
            if (nd) CK(cudaMallocAsync(&wd, nd, st));
            // tiled-permutation tables: one device copy for the call
            std::vector<int32_t> tall;
            for (auto pr : {std::make_pair(&op.px, &op.tpx), std::make_pair(&op.py, &op.tpy),
                            std::make_pair(&op.post, &op.tpost)}) {
                if (pr.first->tl.tn <= 0) continue;
                tall.resize((tall.size() + 3) & ~(size_t)3);   // 16-byte aligned
                pr.first->tl.ttab = (const int32_t *)(uintptr_t)tall.size();   // offset for now
                tall.insert(tall.end(), pr.second->begin(), pr.second->end());
            }
            int32_t *dtab = nullptr;
            if (!tall.empty()) {
                CK(cudaMallocAsync(&dtab, tall.size() * 4, st));
                CK(cudaMemcpyAsync(dtab, tall.data(), tall.size() * 4, cudaMemcpyHostToDevice, st));
                for (PDesc *q : {&op.px, &op.py, &op.post})
                    if (q->tl.tn > 0) q->tl.ttab = dtab + (uintptr_t)q->tl.ttab;
            }
            op.px.out = wx;
            op.py.out = wy;
            op.g.X = wx;
            op.g.Y = wy;
            if (op.has_post) {
                op.g.D = wd;
                op.post.in = wd;
            }
            bool tc = (prec == TN_TF32 || prec == TN_BF16) && dtype == 1 && tc_gemm_supported(op.g);
            int *d_err = nullptr;
            {
                tn_status fs = device_err_flag(&d_err);
                if (fs) return fs;
            }
            launch_permute(op.px, st);
            launch_permute(op.py, st);
            cudaError_t le = cudaSuccess;
            if (tc) le = launch_tc_gemm(op.g, d_err, st);
            else launch_simt_gemm(op.g, st);
            if (op.has_post) launch_permute(op.post, st);
            cudaError_t e2 = cudaGetLastError();
            cudaFreeAsync(wx, st);
            cudaFreeAsync(wy, st);
            if (wd) cudaFreeAsync(wd, st);
            if (dtab) {
                // the pageable source of the table copy must outlive it
                cudaStreamSynchronize(st);
                cudaFreeAsync(dtab, st);
            }
            if (le != cudaSuccess || e2 != cudaSuccess)
                return fail(TN_E_CUDA, std::string("GEMM launch: ") +
                                           cudaGetErrorString(le != cudaSuccess ? le : e2));
            CK(cudaStreamSynchronize(st));
            int herr = 0;
            CK(cudaMemcpy(&herr, d_err, 4, cudaMemcpyDeviceToHost));
            if (herr) {
                CK(cudaMemset(d_err, 0, 4));
                return fail(TN_E_TIMEOUT, "a device-side wait exceeded its time limit");
            }
            return TN_OK;
        }
    }
    int es = dtype == 0 ? 8 : 4;
    // other sum-product contractions without a label summed inside one
    // operand: the batched strided GEMM
    if (semiring == 0) {
        BDesc bd;
        std::vector<int32_t> tab;
        const bool tc_in = prec == TN_TF32 || prec == TN_BF16;
        if (make_bgemm(card, la, false, 0, A, nullptr, lb, false, 0, B, nullptr, lc, false, 0, C,
                       nullptr, 1, es, bd, tab, tc_in)) {
            int32_t *dtab = nullptr;
            void *part = nullptr;
            size_t pb = bgemm_scratch_bytes(bd, es);
            CK(cudaMallocAsync(&dtab, tab.size() * 4, st));
            CK(cudaMemcpyAsync(dtab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
            for (const int32_t **q : {&bd.tag, &bd.tbg, &bd.tcg, &bd.tam, &bd.tcm, &bd.tbn,
                                      &bd.tcn, &bd.tak, &bd.tbk})
                *q = dtab + (intptr_t)*q;
            if (pb) CK(cudaMallocAsync(&part, pb, st));
            tn_status fs = device_err_flag(&bd.err);
            if (fs) return fs;
            if (!tc_in) bd.tc = 0;   // TF32 inputs only when asked
            if (dtype == 0) launch_bgemm<double>(bd, part, st);
            else launch_bgemm<float>(bd, part, st);
            cudaError_t e = cudaGetLastError();
            // the pageable source of the table copy must outlive it
            cudaError_t e2 = cudaStreamSynchronize(st);
            cudaFreeAsync(dtab, st);
            if (part) cudaFreeAsync(part, st);
            if (e != cudaSuccess || e2 != cudaSuccess)
                return fail(TN_E_CUDA, std::string("batched GEMM launch: ") +
                                           cudaGetErrorString(e != cudaSuccess ? e : e2));
            CK(cudaStreamSynchronize(st));
            int herr = 0;
            CK(cudaMemcpy(&herr, bd.err, 4, cudaMemcpyDeviceToHost));
            if (herr) {
                CK(cudaMemset(bd.err, 0, 4));
                return fail(TN_E_TIMEOUT, "a device-side wait exceeded its time limit");
            }
            return TN_OK;
        }
    }
    CDesc d;
    std::string err = make_desc(card, la, false, 0, A, nullptr, lb, false, 0, B, nullptr, lc,
                                false, C, nullptr, nullptr, 1,
                                semiring == 1 ? argmax : nullptr, d);
    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
    size_t sb = contract_scratch_bytes(d, es);
    void *scratch = nullptr;
    if (sb) CK(cudaMallocAsync(&scratch, sb, st));
    if (dtype == 0) launch_contract<double>(d, semiring, scratch, sb, st, nullptr);
    else launch_contract<float>(d, semiring, scratch, sb, st, nullptr);
    cudaError_t e = cudaGetLastError();
    if (scratch) cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return fail(TN_E_CUDA, std::string("contract launch: ") + cudaGetErrorString(e));
    CK(cudaStreamSynchronize(st));
    return TN_OK;
}

// Time every kernel of a PR (task 0) or PR + MAR (task 1) pass one launch at a
// time, accumulated by kernel class over `reps` passes.  out[8][4]: per class
// total milliseconds, launches, algorithmic FLOPs, algorithmic bytes.
static tn_status profile_impl(tn_model *m, int task, int batch, const int32_t *evid,
                              const tn_options *opts, int reps, double *out, int cap,
                              double *steps, int *nsteps);

tn_status tn_profile(tn_model *m, int task, int batch, const int32_t *evid,
                     const tn_options *opts, int reps, double *out) {
    return profile_impl(m, task, batch, evid, opts, reps, out, 0, nullptr, nullptr);
}

tn_status tn_profile_steps(tn_model *m, int task, int batch, const int32_t *evid,
                           const tn_options *opts, int cap, double *steps, int *nsteps) {
    double cls[4 * C_NCLS];
    return profile_impl(m, task, batch, evid, opts, 1, cls, cap, steps, nsteps);
}

static tn_status profile_impl(tn_model *m, int task, int batch, const int32_t *evid,
                              const tn_options *opts, int reps, double *out, int cap,
                              double *steps, int *nsteps) {
    if (!m || !out || batch < 1 || reps < 1 || (task != 0 && task != 1))
        return fail(TN_E_ARG, "bad argument");
    tn_status s = check_evid(m, batch, evid);
    if (s) return s;
    Program *P;
    s = get_program(m, task == 0 ? K_PR : K_MAR, batch, opts, false, &P);
    if (s) return s;
    cudaStream_t st = m->stream;
    s = override_tables(m, nullptr, 0, st);
    if (s) return s;
    size_t eb = (size_t)batch * m->md.nvars * 4;
    if (eb) {
        if (evid) CK(cudaMemcpy(P->d_evid, evid, eb, cudaMemcpyHostToDevice));
        else CK(cudaMemset(P->d_evid, 0xff, eb));
    }
    Prof pr;
    for (int r = 0; r < reps; ++r) {
        if (P->dtype == 0) enqueue_program<double>(m, *P, st, &pr);
        else enqueue_program<float>(m, *P, st, &pr);
    }
    CK(cudaStreamSynchronize(st));
    pr.finish();
    if (steps && nsteps) {
        int n = (int)(pr.rec.size() / 4);
        *nsteps = n;
        for (int i = 0; i < std::min(n, cap); ++i)
            for (int j = 0; j < 4; ++j) steps[4 * i + j] = pr.rec[4 * i + j];
    }
    for (int c = 0; c < C_NCLS; ++c) {
        out[4 * c + 0] = pr.ms[c] / reps;
        out[4 * c + 1] = pr.n[c] / reps;
        out[4 * c + 2] = pr.flops[c] / reps;
        out[4 * c + 3] = pr.bytes[c] / reps;
    }
    CK(cudaGetLastError());
    return check_device_error(m);
}

tn_status tn_program_stats(tn_model *m, int task, int batch, const tn_options *opts,
                           double *out) {
    if (!m || !out || batch < 1 || (task != 0 && task != 1)) return fail(TN_E_ARG, "bad argument");
    Program *P;
    int sub = batch;
    tn_status s = program_fitting(m, task == 0 ? K_PR : K_MAR, batch, opts, false, &P, &sub);
    if (s) return s;
    out[0] = (double)P->arena_elems * P->esz;
    out[1] = (double)P->keep_all_elems * P->esz;
    out[2] = P->ndrop;
    out[3] = P->launches;
    out[4] = P->nlanes;
    out[5] = P->tune.absorb_bps;
    out[6] = P->tune.tuned ? 1 : 0;
    out[7] = sub;
    return TN_OK;
}

double tn_last_device_ms(const tn_model *m) { return m ? m->last_ms : 0.0; }
int64_t tn_last_launch_count(const tn_model *m) { return m ? m->last_launches : 0; }

}  // extern "C"

// Executor and C ABI of libtn.
//
// A task (PR, MAR, MPE, sampling) on a model becomes a Program: the plan of
// the contraction tree (labels, layouts, summed labels per node), one device
// arena holding every tensor the task needs, one buffer of per-item maxima
// for the power-of-two rescaling, and the list of kernel launches.  The
// launches are captured once into a CUDA graph and replayed on every call, so
// a call costs one graph launch plus the copies of its inputs and outputs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "kernels.cuh"
#include "model.h"
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
        if (e_ != cudaSuccess)                                                            \
            return fail(TN_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
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

struct Program {
    int kind = 0, dtype = 0, esz = 8, nbeta = 1;
    bool grads = false;
    Plan plan;
    std::vector<Slot> fwd, adj;
    std::vector<char> adj_beta, need_adj;
    int64_t nmx = 0;
    DevMem mem;
    char *arena = nullptr;
    int64_t arena_elems = 0;
    unsigned long long *mx = nullptr;
    int32_t *am = nullptr;
    std::vector<int64_t> am_off;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
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
    double *d_logz = nullptr, *d_sigma = nullptr, *d_marg = nullptr, *d_grad = nullptr;
    int32_t *d_assign = nullptr;
    int *d_card = nullptr;
    std::vector<CDesc> fdesc, bdesc;
    std::vector<LeafRec> leafrec;   // host copy (external sources patched per call)
    cudaGraphExec_t gexec = nullptr;
    int launches = 0;
    int64_t marg_stride = 0, grad_stride = 0;
    ~Program() {
        if (gexec) cudaGraphExecDestroy(gexec);
    }
};

}  // namespace

struct tn_model {
    ModelData md;
    Tree tree;
    bool has_tree = false;
    std::vector<int> slice_vars;
    double *d_tables = nullptr;
    int *d_flags = nullptr;            // [0]: tables hold logarithms
    bool tables_overridden = false;
    int device = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::map<std::tuple<int, int, int, int>, std::unique_ptr<Program>> progs;
    double last_ms = 0;
    int64_t last_launches = 0;
    ~tn_model() {
        progs.clear();
        if (d_tables) cudaFree(d_tables);
        if (d_flags) cudaFree(d_flags);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

Net model_net(const ModelData &md, bool batched) {
    Net n;
    n.card = md.card;
    for (int f = 0; f < md.nfactors; ++f) {
        n.leaf.push_back(md.scope[f]);
        n.leaf_beta.push_back(0);
    }
    for (int v = 0; v < md.nvars; ++v) {
        n.leaf.push_back({v});
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

// Build (plan, allocate, describe, capture) a program.
tn_status build_program(tn_model *m, const Net &net, const Tree &tree, int kind, int dtype,
                        int nbeta, bool grads, const tn_options *opts, Program &P,
                        const std::vector<LeafRec> *spec = nullptr) {
    P.kind = kind;
    P.dtype = dtype;
    P.esz = (int)elem_bytes(dtype);
    P.nbeta = nbeta;
    P.grads = grads;
    std::string err = build_plan(net, tree, P.plan);
    if (!err.empty()) return fail(TN_E_ORDER, err);
    const Plan &pl = P.plan;
    const int n = tree.nleaves;
    const int NN = 2 * n - 1;
    const bool maxplus = kind == K_MAP || kind == K_MAXNET;
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
    // ---- arena offsets
    OffsetAlloc A;
    for (int id = 0; id < n; ++id) P.fwd[id].off = A.alloc(P.fwd[id].elems);
    for (int id = n; id < NN; ++id) {
        const Node &nd = pl.node[id];
        P.fwd[id].off = A.alloc(P.fwd[id].elems);
        if (!keep_all) {
            A.release(P.fwd[nd.a].off, P.fwd[nd.a].elems);
            A.release(P.fwd[nd.b].off, P.fwd[nd.b].elems);
        }
    }
    if (backward) {
        P.adj[pl.root].off = A.alloc(P.adj[pl.root].elems);
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            for (int c : {nd.a, nd.b})
                if (P.need_adj[c]) P.adj[c].off = A.alloc(P.adj[c].elems);
            A.release(P.adj[id].off, P.adj[id].elems);
        }
    }
    P.arena_elems = A.top;
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
    int64_t budget = opts ? opts->hbm_budget_bytes : 0;
    size_t freeb = 0, totb = 0;
    CK(cudaMemGetInfo(&freeb, &totb));
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
    CK(P.mem.alloc(&P.d_logz, (size_t)nbeta * 8));
    CK(P.mem.alloc(&P.d_sigma, (size_t)nbeta * 8));
    CK(P.mem.alloc(&P.d_card, net.card.size() * 4 + 4));
    CK(cudaMemcpy(P.d_card, net.card.data(), net.card.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemset(P.d_evid, 0xff, (size_t)nbeta * std::max(1, m->md.nvars) * 4));
    // ---- leaf records
    for (int id = 0; id < n; ++id) {
        LeafRec r;
        std::memset(&r, 0, sizeof r);
        if (spec) {
            r = (*spec)[id];
            if (r.kind == LEAF_UNITY) r.beta = pl.node[id].beta;
        } else if (id < (int)m->md.nfactors) {
            r.kind = LEAF_FACTOR;
            r.src = m->md.toff[id];
        } else {
            r.kind = LEAF_UNITY;
            r.var = net.leaf[id].empty() ? 0 : net.leaf[id][0];
            r.beta = pl.node[id].beta;
        }
        r.size = P.fwd[id].per;
        r.dst = P.fwd[id].off;
        r.mx = P.fwd[id].mx;
        P.leafrec.push_back(r);
    }
    P.nleafrec = n;
    // ---- descriptors
    auto mxp = [&](int64_t i) { return maxplus ? nullptr : P.mx + i; };
    size_t scratch = 0;
    for (int id = n; id < NN; ++id) {
        const Node &nd = pl.node[id];
        CDesc d;
        err = make_desc(net.card, pl.node[nd.a].labels, pl.node[nd.a].beta, P.fwd[nd.a].per,
                        (char *)P.arena + P.fwd[nd.a].off * P.esz,
                        mxp(P.fwd[nd.a].mx), pl.node[nd.b].labels, pl.node[nd.b].beta,
                        P.fwd[nd.b].per, (char *)P.arena + P.fwd[nd.b].off * P.esz,
                        mxp(P.fwd[nd.b].mx), nd.labels, nd.beta,
                        (char *)P.arena + P.fwd[id].off * P.esz, mxp(P.fwd[id].mx), &nd.elim,
                        nbeta, maxplus ? P.am + P.am_off[id] : nullptr, d);
        if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
        scratch = std::max(scratch, contract_scratch_bytes(d, P.esz));
        P.fdesc.push_back(d);
    }
    if (backward) {
        for (int id = NN - 1; id >= n; --id) {
            const Node &nd = pl.node[id];
            const Node &na = pl.node[nd.a], &nb = pl.node[nd.b];
            char *cbar = (char *)P.arena + P.adj[id].off * P.esz;
            CDesc d;
            if (P.need_adj[nd.a]) {
                err = make_desc(net.card, nd.labels, P.adj_beta[id], P.adj[id].per, cbar,
                                P.mx + P.adj[id].mx, nb.labels, nb.beta, P.fwd[nd.b].per,
                                (char *)P.arena + P.fwd[nd.b].off * P.esz, P.mx + P.fwd[nd.b].mx,
                                na.labels, P.adj_beta[nd.a],
                                (char *)P.arena + P.adj[nd.a].off * P.esz, P.mx + P.adj[nd.a].mx,
                                nullptr, nbeta, nullptr, d);
                if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                scratch = std::max(scratch, contract_scratch_bytes(d, P.esz));
                P.bdesc.push_back(d);
            }
            if (P.need_adj[nd.b]) {
                err = make_desc(net.card, na.labels, na.beta, P.fwd[nd.a].per,
                                (char *)P.arena + P.fwd[nd.a].off * P.esz, P.mx + P.fwd[nd.a].mx,
                                nd.labels, P.adj_beta[id], P.adj[id].per, cbar,
                                P.mx + P.adj[id].mx, nb.labels, P.adj_beta[nd.b],
                                (char *)P.arena + P.adj[nd.b].off * P.esz, P.mx + P.adj[nd.b].mx,
                                nullptr, nbeta, nullptr, d);
                if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
                scratch = std::max(scratch, contract_scratch_bytes(d, P.esz));
                P.bdesc.push_back(d);
            }
        }
    }
    P.scratch_bytes = scratch;
    if (scratch) CK(P.mem.alloc(&P.scratch, scratch));
    // ---- leaf records to device
    CK(P.mem.alloc(&P.d_leaf, sizeof(LeafRec) * n));
    CK(cudaMemcpy(P.d_leaf, P.leafrec.data(), sizeof(LeafRec) * n, cudaMemcpyHostToDevice));
    // ---- exponent list for log Z
    if (!maxplus) {
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
            if (K > 4096) {
                int64_t rows = P.fwd[id].per;
                if ((double)rows * (double)K > (double)(1LL << 27))
                    return fail(TN_E_UNSUPPORTED,
                                "sampling: a node sums too many labels for its output size");
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

template <typename T>
void enqueue_program(tn_model *m, Program &P, cudaStream_t st) {
    const Plan &pl = P.plan;
    const int n = pl.tree.nleaves, NN = 2 * n - 1;
    const bool maxplus = P.kind == K_MAP || P.kind == K_MAXNET;
    int nl = 0;
    cudaMemsetAsync(P.mx, 0, (size_t)P.nmx * 8, st);
    ++nl;
    launch_leaves<T>(P.d_leaf, P.nleafrec, m->d_tables, P.d_card, m->md.nvars, P.d_evid, P.nbeta,
                     maxplus ? 1 : 0, (T *)P.arena, P.mx, m->d_flags, st);
    ++nl;
    for (auto &d : P.fdesc)
        launch_contract<T>(d, maxplus ? MAXPLUS : SUM, P.scratch, P.scratch_bytes, st, &nl);
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
        for (auto &d : P.bdesc) launch_contract<T>(d, SUM, P.scratch, P.scratch_bytes, st, &nl);
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
    CK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    if (P.dtype == 0) enqueue_program<double>(m, P, m->stream);
    else enqueue_program<float>(m, P, m->stream);
    cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (e != cudaSuccess) return fail(TN_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&P.gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(TN_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return TN_OK;
}

tn_status ensure_device(tn_model *m) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (m->device == dev && m->d_tables && !m->tables_overridden) return TN_OK;
    if (m->device != dev) {
        m->progs.clear();
        if (m->d_tables) cudaFree(m->d_tables);
        m->d_tables = nullptr;
        if (m->stream) cudaStreamDestroy(m->stream);
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
    if (!m->md.tables.empty())
        CK(cudaMemcpy(m->d_tables, m->md.tables.data(), m->md.tables.size() * 8,
                      cudaMemcpyHostToDevice));
    m->tables_overridden = false;
    return TN_OK;
}

int dtype_of(tn_prec p) { return p == TN_FP64 ? 0 : 1; }

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
    auto key = std::make_tuple(kind, dtype, nbeta, grads ? 1 : 0);
    auto it = m->progs.find(key);
    if (it != m->progs.end()) {
        *out = it->second.get();
        return TN_OK;
    }
    auto P = std::make_unique<Program>();
    Net net = model_net(m->md, nbeta > 1);
    s = build_program(m, net, m->tree, kind, dtype, nbeta, grads, opts, *P);
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

// Run a captured program: copy the evidence in, replay the graph, time it.
tn_status run_program(tn_model *m, Program &P, const int32_t *evid, bool evid_on_device,
                      cudaStream_t st) {
    size_t eb = (size_t)P.nbeta * m->md.nvars * 4;
    if (eb) {
        if (evid)
            CK(cudaMemcpyAsync(P.d_evid, evid, eb,
                               evid_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        else
            CK(cudaMemsetAsync(P.d_evid, 0xff, eb, st));
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
    return TN_OK;
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
    if (nslice > 0) {
        if (!slice_vars) return fail(TN_E_ARG, "NULL slice variables");
        for (int i = 0; i < nslice; ++i)
            if (slice_vars[i] < 0 || slice_vars[i] >= m->md.nvars)
                return fail(TN_E_ARG, "slice variable out of range");
        return fail(TN_E_UNSUPPORTED, "slicing is not supported by this build");
    }
    m->tree = t;
    m->has_tree = true;
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
    if (method < 0 || method > 1) return fail(TN_E_ARG, "unknown method");
    Tree t = optimize_tree(model_net(m->md, false), method, restarts, seed);
    std::copy(t.left.begin(), t.left.end(), left);
    std::copy(t.right.begin(), t.right.end(), right);
    return TN_OK;
}

tn_status tn_tree_stats(const tn_model *m, int batch, tn_prec prec, double *out) {
    if (!m || !out || batch < 1) return fail(TN_E_ARG, "bad argument");
    Net net = model_net(m->md, batch > 1);
    Tree t = m->has_tree ? m->tree : greedy_tree(model_net(m->md, false));
    Plan p;
    std::string err = build_plan(net, t, p);
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
    out[0] = mul > 0 ? std::log2(mul) : 0;
    out[1] = sc;
    out[2] = bytes > 0 ? std::log2(bytes / es) : 0;
    out[3] = n - 1;
    out[4] = 2 * mul;
    out[5] = bytes;
    return TN_OK;
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
    tn_status s = get_program(m, K_PR, batch, opts, false, &P);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, tables_dev, is_log, st);
    if (s) return s;
    s = run_program(m, *P, evid, evid_dev, st);
    if (s) return s;
    CK(cudaMemcpyAsync(logz, P->d_logz, (size_t)batch * 8,
                       logz_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
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
    tn_status s = get_program(m, K_MAR, batch, opts, grad != nullptr, &P);
    if (s) return s;
    cudaStream_t st = stream_of(m, opts);
    s = override_tables(m, tables_dev, is_log, st);
    if (s) return s;
    s = run_program(m, *P, evid, dev, st);
    if (s) return s;
    cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(logz, P->d_logz, (size_t)batch * 8, k, st));
    CK(cudaMemcpyAsync(marg, P->d_marg, (size_t)batch * P->marg_stride * 8, k, st));
    if (grad) CK(cudaMemcpyAsync(grad, P->d_grad, (size_t)batch * P->grad_stride * 8, k, st));
    CK(cudaStreamSynchronize(st));
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

tn_status tn_mar_dev(tn_model *m, int batch, const int32_t *evid, const double *factor_tables,
                     int tables_are_log, const tn_options *opts, double *logz, double *marg,
                     double *grad) {
    return mar_common(m, batch, evid, true, factor_tables, tables_are_log, opts, logz, marg,
                      grad);
}

tn_status tn_map(tn_model *m, const int32_t *evid, const tn_options *opts, int32_t *assign,
                 double *logp) {
    if (!m || !assign || !logp) return fail(TN_E_ARG, "bad argument");
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
    s = run_program(m, *P, evid, false, st);
    if (s) return s;
    double lz;
    CK(cudaMemcpy(&lz, P->d_logz, 8, cudaMemcpyDeviceToHost));
    if (!(lz > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
    if (n == 0) return TN_OK;
    int8_t *d_out = nullptr;
    CK(cudaMallocAsync(&d_out, (size_t)n * m->md.nvars, st));
    CK(cudaEventRecord(m->ev0, st));
    {
        // cumulative tables of the nodes with large summed spaces
        int64_t coff = 0;
        for (auto &c : P->cdf_nodes) {
            if (P->dtype == 0) launch_cdf_rows<double>(c.first, c.second, P->cdf + coff, st);
            else launch_cdf_rows<float>(c.first, c.second, P->cdf + coff, st);
            coff += c.second * c.first.ktotal;
        }
    }
    if (P->dtype == 0)
        launch_sample<double>(P->d_meta, P->nmeta, (const double *)P->arena, P->cdf, P->d_evid,
                              m->md.nvars, n, seed, d_out, st);
    else
        launch_sample<float>(P->d_meta, P->nmeta, (const float *)P->arena, P->cdf, P->d_evid,
                             m->md.nvars, n, seed, d_out, st);
    CK(cudaEventRecord(m->ev1, st));
    CK(cudaMemcpyAsync(samples, d_out, (size_t)n * m->md.nvars, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(d_out, st));
    CK(cudaStreamSynchronize(st));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    m->last_ms += ms;
    CK(cudaGetLastError());
    return TN_OK;
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
    Program P2;
    s = build_program(m, net2, t2, K_MAP, dtype, 1, false, opts, P2, &spec2);
    if (s) return s;
    s = capture_program(m, P2);
    if (s) return s;
    s = run_program(m, P2, evid, false, st);
    if (s) return s;
    launches += P2.launches;
    double lp;
    std::vector<int32_t> x(md.nvars);
    CK(cudaMemcpyAsync(&lp, P2.d_logz, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(x.data(), P2.d_assign, (size_t)md.nvars * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *logp = lp + lconst;
    for (int i = 0; i < nq; ++i) assign[i] = x[query[i]];
    m->last_launches = launches;
    if (!(lp > -INFINITY)) return fail(TN_E_ARG, "p(e) = 0");
    return TN_OK;
}

// One pairwise contraction on caller-provided device buffers.
tn_status tn_contract_dev(int nlabels, const int *sizes, int na, const int *labels_a,
                          const void *A, int nb, const int *labels_b, const void *B, int nc,
                          const int *labels_c, void *C, int semiring, int dtype, tn_prec prec,
                          int32_t *argmax, void *cuda_stream) {
    (void)prec;
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
    CDesc d;
    std::string err = make_desc(card, la, false, 0, A, nullptr, lb, false, 0, B, nullptr, lc,
                                false, C, nullptr, nullptr, 1,
                                semiring == 1 ? argmax : nullptr, d);
    if (!err.empty()) return fail(TN_E_UNSUPPORTED, err);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int es = dtype == 0 ? 8 : 4;
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

double tn_last_device_ms(const tn_model *m) { return m ? m->last_ms : 0.0; }
int64_t tn_last_launch_count(const tn_model *m) { return m ? m->last_launches : 0; }

}  // extern "C"

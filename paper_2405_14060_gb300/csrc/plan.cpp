// Contraction-tree planning (host): tree validation, per-node label
// classification and layouts, complexity accounting, and order search
// (greedy pair merging, elimination orders, randomised min-fill).
//
// A pairwise contraction keeps a label iff the label still occurs outside the
// subtree or is an output label; every other label of its operands is summed
// (max-plus: maximised) there (Sec. Tensor networks: "each internal node
// results from contracting two child tensors and summing out any indices not
// needed for later operations").
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <queue>
#include <random>
#include <set>
#include <unordered_map>

#include "tn_internal.h"

namespace tn {

double log2_size(const Net &net, const Labels &l) {
    double s = 0;
    for (int v : l) s += std::log2((double)net.card[v]);
    return s;
}

std::string validate_tree(const Tree &t) {
    int n = t.nleaves;
    if (n < 1) return "tree has no leaves";
    if ((int)t.left.size() != n - 1 || (int)t.right.size() != n - 1)
        return "tree must have nleaves-1 internal nodes";
    std::vector<char> used(2 * n - 1, 0);
    for (int i = 0; i < n - 1; ++i) {
        int me = n + i;
        for (int c : {t.left[i], t.right[i]}) {
            if (c < 0 || c >= me) return "child id out of range or not earlier than its parent";
            if (used[c]) return "a tensor is contracted twice";
            used[c] = 1;
        }
        if (t.left[i] == t.right[i]) return "a node contracts a tensor with itself";
    }
    for (int id = 0; id < 2 * n - 2; ++id)
        if (!used[id]) return "a tensor is never contracted";
    return "";
}

// Sparse label multiset: sorted (label, count) pairs.
using LCount = std::vector<std::pair<int, int>>;

static LCount merge_counts(const LCount &x, const LCount &y) {
    LCount r;
    r.reserve(x.size() + y.size());
    size_t i = 0, j = 0;
    while (i < x.size() || j < y.size()) {
        if (j == y.size() || (i < x.size() && x[i].first < y[j].first)) r.push_back(x[i++]);
        else if (i == x.size() || y[j].first < x[i].first) r.push_back(y[j++]);
        else { r.push_back({x[i].first, x[i].second + y[j].second}); ++i; ++j; }
    }
    return r;
}

std::string build_plan(const Net &net, const Tree &tree, Plan &plan, int64_t gemm_min) {
    std::string err = validate_tree(tree);
    if (!err.empty()) return err;
    int n = tree.nleaves;
    if ((int)net.leaf.size() != n) return "tree leaf count does not match the network";
    plan.net = net;
    plan.tree = tree;
    plan.node.assign(2 * n - 1, Node());
    std::vector<int> total(net.card.size(), 0);
    std::vector<char> isout(net.card.size(), 0);
    for (int v : net.out) isout[v] = 1;
    std::vector<LCount> cnt(2 * n - 1);
    for (int i = 0; i < n; ++i) {
        Node &nd = plan.node[i];
        nd.labels = net.leaf[i];
        nd.beta = net.leaf_beta.empty() ? false : net.leaf_beta[i];
        nd.size = 1;
        for (int v : nd.labels) {
            nd.size *= net.card[v];
            total[v]++;
        }
        Labels s = nd.labels;
        std::sort(s.begin(), s.end());
        for (size_t k = 0; k < s.size(); ++k) {
            if (k && s[k] == s[k - 1]) return "a leaf repeats a label";
            cnt[i].push_back({s[k], 1});
        }
    }
    double tot_mul = 0, tot_rw = 0, sc = 0;
    for (int i = 0; i < n - 1; ++i) {
        int me = n + i;
        int x = tree.left[i], y = tree.right[i];
        Node &nd = plan.node[me];
        plan.node[x].parent = me;
        plan.node[y].parent = me;
        cnt[me] = merge_counts(cnt[x], cnt[y]);
        // keep rule
        std::vector<char> keep_l;
        std::set<int> kept;
        for (auto &p : cnt[me])
            if (p.second < total[p.first] || isout[p.first]) kept.insert(p.first);
        // a = larger operand (its layout is kept), b = smaller
        int a = x, b = y;
        if (plan.node[y].size > plan.node[x].size) std::swap(a, b);
        nd.a = a;
        nd.b = b;
        const Labels &la = plan.node[a].labels, &lb = plan.node[b].labels;
        std::set<int> sa(la.begin(), la.end());
        // output layout: labels new to C from b (in b's order), then a's kept
        // labels in a's order
        nd.labels.clear();
        for (int v : lb)
            if (!sa.count(v) && kept.count(v)) nd.labels.push_back(v);
        for (int v : la)
            if (kept.count(v)) nd.labels.push_back(v);
        nd.beta = plan.node[a].beta || plan.node[b].beta;
        // GEMM form: groups bt (in both, kept), m (row operand only, kept),
        // n (column operand only, kept), k (in both, summed); the operand
        // holding the batch label goes on the row side so that the label
        // stays outermost in C = [bt, m, n].
        if (gemm_min > 0) {
            int ga = a, gb = b;
            if (plan.node[b].beta && !plan.node[a].beta) std::swap(ga, gb);
            const Labels &xa = plan.node[ga].labels, &xb = plan.node[gb].labels;
            std::set<int> sxa(xa.begin(), xa.end()), sxb(xb.begin(), xb.end());
            Labels gbt, gm, gn, gk;
            bool onesided = false;
            for (int v : xa) {
                if (kept.count(v)) (sxb.count(v) ? gbt : gm).push_back(v);
                else if (sxb.count(v)) gk.push_back(v);
                else onesided = true;
            }
            for (int v : xb) {
                if (kept.count(v) && !sxa.count(v)) gn.push_back(v);
                else if (!kept.count(v) && !sxa.count(v)) onesided = true;
            }
            auto prod = [&](const Labels &l) {
                int64_t p = 1;
                for (int v : l) p *= net.card[v];
                return p;
            };
            if (!onesided && prod(gm) >= gemm_min && prod(gn) >= gemm_min &&
                prod(gk) >= gemm_min) {
                nd.gemm = true;
                nd.ga = ga;
                nd.gb = gb;
                nd.gbt = gbt;
                nd.gm = gm;
                nd.gn = gn;
                nd.labels.clear();
                for (int v : gbt) nd.labels.push_back(v);
                for (int v : gm) nd.labels.push_back(v);
                for (int v : gn) nd.labels.push_back(v);
            }
        }
        nd.size = 1;
        for (int v : nd.labels) nd.size *= net.card[v];
        // eliminated labels in kernel order: a's order, then b-only labels
        nd.elim.clear();
        if (nd.gemm) {
            for (int v : plan.node[nd.ga].labels)
                if (!kept.count(v)) nd.elim.push_back(v);
        } else {
            for (int v : la)
                if (!kept.count(v)) nd.elim.push_back(v);
            for (int v : lb)
                if (!sa.count(v) && !kept.count(v)) nd.elim.push_back(v);
        }
        double mul = 1;
        for (auto &p : cnt[me]) mul *= net.card[p.first];
        nd.muladds = mul;
        tot_mul += mul;
        tot_rw += (double)plan.node[a].size + (double)plan.node[b].size + (double)nd.size;
        sc = std::max(sc, std::log2((double)nd.size));
        // drop eliminated labels from the count list
        LCount c2;
        for (auto &p : cnt[me])
            if (kept.count(p.first)) c2.push_back(p);
        cnt[me].swap(c2);
        cnt[x].clear();
        cnt[y].clear();
    }
    plan.root = 2 * n - 2;
    // depths (root 0)
    for (int id = 2 * n - 2; id >= 0; --id) {
        int p = plan.node[id].parent;
        plan.node[id].depth = p < 0 ? 0 : plan.node[p].depth + 1;
    }
    plan.total_muladds = tot_mul;
    plan.total_rw_entries = tot_rw;
    plan.tc_log2 = tot_mul > 0 ? std::log2(tot_mul) : 0;
    plan.rw_log2 = tot_rw > 0 ? std::log2(tot_rw) : 0;
    plan.sc_log2 = sc;
    return "";
}

// ------------------------------------------------------------------ greedy
//
// Repeatedly contract the pair of connected tensors (sharing a label) whose
// result grows least, measured as log2|C| - log2(|A| + |B|); ties go to the
// pair with the smaller (min id, max id).  Tensors with no shared label are
// merged last, two smallest first.

namespace {
struct Frontier {
    const Net &net;
    std::vector<Labels> lab;          // sorted labels of each tensor id
    std::vector<char> alive;
    std::vector<int> count;           // alive tensors holding each label
    std::vector<std::set<int>> holders;
    std::vector<char> isout;
    explicit Frontier(const Net &n) : net(n) {
        int L = (int)n.card.size();
        count.assign(L, 0);
        holders.assign(L, {});
        isout.assign(L, 0);
        for (int v : n.out) isout[v] = 1;
        for (size_t i = 0; i < n.leaf.size(); ++i) {
            Labels s = n.leaf[i];
            std::sort(s.begin(), s.end());
            lab.push_back(s);
            alive.push_back(1);
            for (int v : s) {
                count[v]++;
                holders[v].insert((int)i);
            }
        }
    }
    double lsize(int id) const {
        double s = 0;
        for (int v : lab[id]) s += std::log2((double)net.card[v]);
        return s;
    }
    Labels merged(int x, int y) const {
        Labels u;
        std::set_union(lab[x].begin(), lab[x].end(), lab[y].begin(), lab[y].end(),
                       std::back_inserter(u));
        Labels r;
        for (int v : u) {
            int inside = (std::binary_search(lab[x].begin(), lab[x].end(), v) ? 1 : 0) +
                         (std::binary_search(lab[y].begin(), lab[y].end(), v) ? 1 : 0);
            if (count[v] > inside || isout[v]) r.push_back(v);
        }
        return r;
    }
    int merge(int x, int y) {
        Labels r = merged(x, y);
        int id = (int)lab.size();
        for (int v : lab[x]) { count[v]--; holders[v].erase(x); }
        for (int v : lab[y]) { count[v]--; holders[v].erase(y); }
        for (int v : r) { count[v]++; holders[v].insert(id); }
        alive[x] = alive[y] = 0;
        lab.push_back(r);
        alive.push_back(1);
        return id;
    }
    std::set<int> neighbours(int id) const {
        std::set<int> s;
        for (int v : lab[id])
            for (int w : holders[v])
                if (w != id) s.insert(w);
        return s;
    }
};

void record(Tree &t, int n, int x, int y, int id) {
    (void)n;
    (void)id;
    t.left.push_back(x);
    t.right.push_back(y);
}

// merge every remaining alive tensor, two smallest first
void merge_rest(Frontier &F, Tree &t) {
    using E = std::pair<double, int>;
    std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
    for (size_t i = 0; i < F.alive.size(); ++i)
        if (F.alive[i]) pq.push({F.lsize((int)i), (int)i});
    while (pq.size() > 1) {
        int x = pq.top().second; pq.pop();
        int y = pq.top().second; pq.pop();
        int id = F.merge(std::min(x, y), std::max(x, y));
        record(t, 0, std::min(x, y), std::max(x, y), id);
        pq.push({F.lsize(id), id});
    }
}
}  // namespace

Tree greedy_tree(const Net &net) {
    Frontier F(net);
    Tree t;
    t.nleaves = (int)net.leaf.size();
    struct Cand {
        double cost;
        int x, y;
        bool operator>(const Cand &o) const {
            if (cost != o.cost) return cost > o.cost;
            if (x != o.x) return x > o.x;
            return y > o.y;
        }
    };
    std::vector<int> ver(2 * net.leaf.size() + 1, 0);
    struct Entry {
        Cand c;
        int vx, vy;
        bool operator>(const Entry &o) const { return c > o.c; }
    };
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    auto cost = [&](int x, int y) {
        Labels r = F.merged(x, y);
        double lc = 0;
        for (int v : r) lc += std::log2((double)net.card[v]);
        double la = F.lsize(x), lb = F.lsize(y);
        double m = std::max(la, lb);
        double lsum = m + std::log2(std::exp2(la - m) + std::exp2(lb - m));
        return lc - lsum;
    };
    auto push_pair = [&](int x, int y) {
        if (x > y) std::swap(x, y);
        pq.push({{cost(x, y), x, y}, ver[x], ver[y]});
    };
    for (size_t i = 0; i < net.leaf.size(); ++i)
        for (int w : F.neighbours((int)i))
            if ((int)i < w) push_pair((int)i, w);
    int remaining = (int)net.leaf.size();
    while (remaining > 1 && !pq.empty()) {
        Entry e = pq.top();
        pq.pop();
        int x = e.c.x, y = e.c.y;
        if (!F.alive[x] || !F.alive[y] || ver[x] != e.vx || ver[y] != e.vy) continue;
        std::set<int> nb = F.neighbours(x);
        for (int w : F.neighbours(y)) nb.insert(w);
        int id = F.merge(x, y);
        record(t, 0, x, y, id);
        --remaining;
        if ((int)ver.size() <= id) ver.resize(id + 1, 0);
        nb.erase(x);
        nb.erase(y);
        // costs of pairs touching the changed labels' holders are stale
        std::set<int> touched = nb;
        for (int w : nb)
            for (int u : F.neighbours(w)) touched.insert(u);
        for (int w : touched) ver[w]++;
        for (int w : touched) {
            if (!F.alive[w]) continue;
            for (int u : F.neighbours(w)) push_pair(w, u);
        }
        for (int u : F.neighbours(id)) push_pair(id, u);
    }
    merge_rest(F, t);
    return t;
}

Tree tree_from_elimination(const Net &net, const std::vector<int> &order_in) {
    Frontier F(net);
    Tree t;
    t.nleaves = (int)net.leaf.size();
    int L = (int)net.card.size();
    std::vector<char> listed(L, 0);
    std::vector<int> order;
    for (int v : order_in)
        if (v >= 0 && v < L && !listed[v]) { listed[v] = 1; order.push_back(v); }
    for (int v = 0; v < L; ++v)
        if (!listed[v]) order.push_back(v);
    using E = std::pair<double, int>;
    for (int v : order) {
        if (F.isout[v]) continue;
        std::priority_queue<E, std::vector<E>, std::greater<E>> pq;
        for (int w : F.holders[v]) pq.push({F.lsize(w), w});
        while (pq.size() > 1) {
            int x = pq.top().second; pq.pop();
            int y = pq.top().second; pq.pop();
            int a = std::min(x, y), b = std::max(x, y);
            int id = F.merge(a, b);
            record(t, 0, a, b, id);
            pq.push({F.lsize(id), id});
        }
    }
    merge_rest(F, t);
    return t;
}

// Randomised min-fill (method 1) / min-degree (odd restarts) elimination
// orders on the interaction graph of the network; ties broken at random.
static std::vector<int> heuristic_order(const Net &net, bool minfill, std::mt19937_64 &rng) {
    int L = (int)net.card.size();
    std::vector<std::vector<char>> adj(L, std::vector<char>(L, 0));
    std::vector<char> present(L, 0), isout(L, 0);
    for (int v : net.out) isout[v] = 1;
    for (auto &lab : net.leaf) {
        for (int v : lab) present[v] = 1;
        for (int u : lab)
            for (int w : lab)
                if (u != w) adj[u][w] = 1;
    }
    std::vector<char> gone(L, 0);
    std::vector<int> order;
    std::vector<int> nb;
    int want = 0;
    for (int v = 0; v < L; ++v)
        if (present[v] && !isout[v]) ++want;
    std::uniform_real_distribution<double> U(0, 1);
    while ((int)order.size() < want) {
        int best = -1;
        double bscore = 0;
        for (int v = 0; v < L; ++v) {
            if (!present[v] || isout[v] || gone[v]) continue;
            nb.clear();
            for (int u = 0; u < L; ++u)
                if (!gone[u] && adj[v][u]) nb.push_back(u);
            double score;
            if (minfill) {
                long fill = 0;
                for (size_t i = 0; i < nb.size(); ++i)
                    for (size_t j = i + 1; j < nb.size(); ++j)
                        if (!adj[nb[i]][nb[j]]) ++fill;
                score = (double)fill;
            } else {
                double w = std::log2((double)net.card[v]);
                for (int u : nb) w += std::log2((double)net.card[u]);
                score = w;
            }
            score += 0.5 * U(rng);   // random tie-breaking (scores are integers / sums)
            if (best < 0 || score < bscore) { best = v; bscore = score; }
        }
        nb.clear();
        for (int u = 0; u < L; ++u)
            if (!gone[u] && adj[best][u]) nb.push_back(u);
        for (int a : nb)
            for (int c : nb)
                if (a != c) adj[a][c] = 1;
        gone[best] = 1;
        order.push_back(best);
    }
    return order;
}

// ------------------------------------------------------- annealed tree
//
// Simulated annealing over contraction trees (local rotations of the binary
// tree, in the spirit of the tree-annealing order finders the paper cites for
// its hyper-optimised orders).  A node's labels are computed from two bitsets:
// U(n), the labels of the leaves under n (bottom-up), and O(n), the labels
// of every leaf outside n (top-down: O(child) = U(sibling) | O(parent)); then
// L(n) = U(n) & O(n).  The objective is
//   log2(sum over nodes of the multiply-add count)  +  w * max(0, sc - target).
namespace {
struct SATree {
    int nl = 0, W = 0;                 // leaves, 64-bit words per bitset
    std::vector<int> ch0, ch1, par;    // per node id (leaves: -1 children)
    std::vector<uint64_t> U, O;        // bitsets, node-major
    std::vector<double> lw;            // log2 card per label
    std::vector<uint64_t> outbits;
    int root = -1;
};

double popw(const uint64_t *b, int W, const std::vector<double> &lw) {
    double s = 0;
    for (int w = 0; w < W; ++w) {
        uint64_t x = b[w];
        while (x) {
            int i = __builtin_ctzll(x);
            s += lw[w * 64 + i];
            x &= x - 1;
        }
    }
    return s;
}

// recompute all bitsets; returns (log2 total multiply-adds, sc)
std::pair<double, double> sa_eval(SATree &T, std::vector<int> &post) {
    const int W = T.W;
    int NN = (int)T.ch0.size();
    // post-order
    post.clear();
    std::vector<int> stack{T.root};
    std::vector<char> seen(NN, 0);
    while (!stack.empty()) {
        int v = stack.back();
        if (v < T.nl || seen[v]) {
            stack.pop_back();
            post.push_back(v);
            continue;
        }
        seen[v] = 1;
        stack.push_back(T.ch1[v]);
        stack.push_back(T.ch0[v]);
    }
    for (int v : post) {
        if (v < T.nl) continue;
        uint64_t *u = &T.U[(size_t)v * W];
        const uint64_t *a = &T.U[(size_t)T.ch0[v] * W], *b = &T.U[(size_t)T.ch1[v] * W];
        for (int w = 0; w < W; ++w) u[w] = a[w] | b[w];
    }
    for (int w = 0; w < W; ++w) T.O[(size_t)T.root * W + w] = T.outbits[w];
    double maxtc = -1e300, sc = 0;
    std::vector<double> terms;
    std::vector<uint64_t> tmp(W), la(W), lb(W);
    for (int i = (int)post.size() - 1; i >= 0; --i) {
        int v = post[i];
        if (v < T.nl) continue;
        int a = T.ch0[v], b = T.ch1[v];
        const uint64_t *Ov = &T.O[(size_t)v * W];
        for (int w = 0; w < W; ++w) {
            T.O[(size_t)a * W + w] = T.U[(size_t)b * W + w] | Ov[w];
            T.O[(size_t)b * W + w] = T.U[(size_t)a * W + w] | Ov[w];
        }
        for (int w = 0; w < W; ++w) {
            la[w] = T.U[(size_t)a * W + w] & T.O[(size_t)a * W + w];
            lb[w] = T.U[(size_t)b * W + w] & T.O[(size_t)b * W + w];
            tmp[w] = la[w] | lb[w];
        }
        double c = popw(tmp.data(), W, T.lw);
        terms.push_back(c);
        maxtc = std::max(maxtc, c);
        for (int w = 0; w < W; ++w) tmp[w] = T.U[(size_t)v * W + w] & Ov[w];
        sc = std::max(sc, popw(tmp.data(), W, T.lw));
    }
    double s = 0;
    for (double c : terms) s += std::exp2(c - maxtc);
    return {maxtc + std::log2(s), sc};
}
}  // namespace

namespace {
// The annealer's state for a tree in tn_set_order's form (leaf bitsets set,
// U and O of internal nodes still to be computed by sa_eval).
void sa_init(const Net &net, const Tree &start, SATree &T) {
    T.nl = (int)net.leaf.size();
    int L = (int)net.card.size();
    T.W = (L + 63) / 64;
    int NN = 2 * T.nl - 1;
    T.ch0.assign(NN, -1);
    T.ch1.assign(NN, -1);
    T.par.assign(NN, -1);
    for (int i = 0; i < T.nl - 1; ++i) {
        T.ch0[T.nl + i] = start.left[i];
        T.ch1[T.nl + i] = start.right[i];
        T.par[start.left[i]] = T.nl + i;
        T.par[start.right[i]] = T.nl + i;
    }
    T.root = NN - 1;
    T.U.assign((size_t)NN * T.W, 0);
    T.O.assign((size_t)NN * T.W, 0);
    T.lw.assign((size_t)T.W * 64, 0.0);
    for (int v = 0; v < L; ++v) T.lw[v] = std::log2((double)net.card[v]);
    T.outbits.assign(T.W, 0);
    for (int v : net.out) T.outbits[v / 64] |= 1ull << (v % 64);
    for (int i = 0; i < T.nl; ++i)
        for (int v : net.leaf[i]) T.U[(size_t)i * T.W + v / 64] |= 1ull << (v % 64);
}

// The tree with children b0 / b1 (root 2 nl - 2) renumbered in post-order.
Tree sa_renumber(int nl, const std::vector<int> &b0, const std::vector<int> &b1) {
    const int NN = 2 * nl - 1;
    Tree t;
    t.nleaves = nl;
    std::vector<int> id(NN, -1);
    for (int i = 0; i < nl; ++i) id[i] = i;
    std::vector<int> stack{NN - 1};
    std::vector<char> seen(NN, 0);
    std::vector<int> order;
    while (!stack.empty()) {
        int v = stack.back();
        if (v < nl || seen[v]) {
            stack.pop_back();
            if (v >= nl) order.push_back(v);
            continue;
        }
        seen[v] = 1;
        stack.push_back(b1[v]);
        stack.push_back(b0[v]);
    }
    int next = nl;
    for (int v : order) id[v] = next++;
    t.left.resize(nl - 1);
    t.right.resize(nl - 1);
    for (int v : order) {
        int k = id[v] - nl;
        t.left[k] = id[b0[v]];
        t.right[k] = id[b1[v]];
    }
    return t;
}
}  // namespace

Tree anneal_tree(const Net &net, const Tree &start, int iters, uint64_t seed, double sc_target) {
    SATree T;
    sa_init(net, start, T);
    const int NN = 2 * T.nl - 1;
    std::vector<int> post;
    auto obj = [&](std::pair<double, double> r) {
        return r.first + 4.0 * std::max(0.0, r.second - sc_target);
    };
    auto cur = sa_eval(T, post);
    double fcur = obj(cur);
    double fbest = fcur;
    std::vector<int> b0 = T.ch0, b1 = T.ch1, bp = T.par;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U01(0, 1);
    std::vector<int> internal;
    for (int v = T.nl; v < NN; ++v) internal.push_back(v);
    for (int it = 0; it < iters; ++it) {
        double beta = 0.5 + 30.0 * it / std::max(1, iters);
        // rotation at node p whose child c (internal) has children x, y:
        // p(c(x, y), z) -> p(c(x, z), y)  or  p(c(y, z), x)
        int p = internal[rng() % internal.size()];
        int side = rng() & 1;
        int c = side ? T.ch1[p] : T.ch0[p];
        if (c < T.nl) continue;
        int z = side ? T.ch0[p] : T.ch1[p];
        int pick = rng() & 1;
        int x = pick ? T.ch1[c] : T.ch0[c];   // stays in c
        int y = pick ? T.ch0[c] : T.ch1[c];   // moves up to p
        // apply
        T.ch0[c] = x;
        T.ch1[c] = z;
        T.par[z] = c;
        if (side) T.ch0[p] = y;
        else T.ch1[p] = y;
        T.par[y] = p;
        auto nxt = sa_eval(T, post);
        double fn = obj(nxt);
        if (fn <= fcur || U01(rng) < std::exp(-beta * (fn - fcur))) {
            fcur = fn;
            cur = nxt;
            if (fn < fbest) {
                fbest = fn;
                b0 = T.ch0;
                b1 = T.ch1;
                bp = T.par;
            }
        } else {
            // undo
            if (side) T.ch0[p] = z;
            else T.ch1[p] = z;
            T.par[z] = p;
            T.ch0[c] = pick ? y : x;
            T.ch1[c] = pick ? x : y;
            T.par[x] = c;
            T.par[y] = c;
        }
    }
    return sa_renumber(T.nl, b0, b1);
}

// The same rotations and objective, evaluated incrementally, with a colder
// schedule (inverse temperature 10 -> 200: the many more moves would
// otherwise wander far from the starting tree at the hot end).  Rotating
// p(c(x, y), z) into p(c(x, z), y) keeps the leaf set under p, x, y and z, so
// U of every node but c is unchanged, and so is O of x, y and z:
// O(x) = U(y) | U(z) | O(p) before and after (likewise for y and z), hence
// for all their descendants.  Only c's labels change, and with them only the
// costs of c and p: a move costs a few bitset words instead of a pass over
// the tree.  The sum of 2^cost is kept relative to a reference exponent (and
// recomputed now and then against drift); the space term comes from a count
// of node sizes.
Tree anneal_tree_fast(const Net &net, const Tree &start, int64_t iters, uint64_t seed,
                      double sc_target) {
    SATree T;
    sa_init(net, start, T);
    const int NN = 2 * T.nl - 1, W = T.W, nl = T.nl;
    std::vector<int> post;
    sa_eval(T, post);
    std::vector<uint64_t> Lb((size_t)NN * W);
    for (size_t i = 0; i < Lb.size(); ++i) Lb[i] = T.U[i] & T.O[i];
    auto Lof = [&](int v) { return &Lb[(size_t)v * W]; };
    std::vector<uint64_t> tmp(W);
    auto cost_of = [&](const uint64_t *a, const uint64_t *b) {
        for (int w = 0; w < W; ++w) tmp[w] = a[w] | b[w];
        return popw(tmp.data(), W, T.lw);
    };
    std::vector<double> cost(NN, 0.0), size(NN, 0.0);
    auto key = [](double v) { return (int64_t)std::llround(v * 1048576.0); };
    std::map<int64_t, int> sizes;   // node sizes (log2, fixed point) -> count
    double ref = 0;
    for (int v = nl; v < NN; ++v) {
        cost[v] = cost_of(Lof(T.ch0[v]), Lof(T.ch1[v]));
        size[v] = popw(Lof(v), W, T.lw);
        sizes[key(size[v])]++;
        ref = std::max(ref, cost[v]);
    }
    double S = 0;
    auto resum = [&]() {
        ref = 0;
        for (int v = nl; v < NN; ++v) ref = std::max(ref, cost[v]);
        S = 0;
        for (int v = nl; v < NN; ++v) S += std::exp2(cost[v] - ref);
    };
    resum();
    auto obj = [&](double Sv, double sc) {
        return ref + std::log2(std::max(Sv, 1e-300)) + 4.0 * std::max(0.0, sc - sc_target);
    };
    auto sc_now = [&]() { return (double)sizes.rbegin()->first / 1048576.0; };
    double fcur = obj(S, sc_now()), fbest = fcur;
    std::vector<int> b0 = T.ch0, b1 = T.ch1;
    std::mt19937_64 rng(seed);
    std::uniform_real_distribution<double> U01(0, 1);
    std::vector<uint64_t> nu(W), no(W), nlc(W);
    int64_t since = 0;
    for (int64_t it = 0; it < iters; ++it) {
        const double beta = 10.0 + 190.0 * (double)it / (double)std::max<int64_t>(1, iters);
        const int p = nl + (int)(rng() % (uint64_t)(nl - 1));
        const int side = rng() & 1;
        const int c = side ? T.ch1[p] : T.ch0[p];
        if (c < nl) continue;
        const int z = side ? T.ch0[p] : T.ch1[p];
        const int pick = rng() & 1;
        const int x = pick ? T.ch1[c] : T.ch0[c];   // stays under c
        const int y = pick ? T.ch0[c] : T.ch1[c];   // moves up to p
        const uint64_t *Ux = &T.U[(size_t)x * W], *Uy = &T.U[(size_t)y * W];
        const uint64_t *Uz = &T.U[(size_t)z * W], *Op = &T.O[(size_t)p * W];
        for (int w = 0; w < W; ++w) {
            nu[w] = Ux[w] | Uz[w];
            no[w] = Uy[w] | Op[w];
            nlc[w] = nu[w] & no[w];
        }
        const double cc = cost_of(Lof(x), Lof(z)), cp = cost_of(nlc.data(), Lof(y));
        const double sz = popw(nlc.data(), W, T.lw);
        const double Sn = S - std::exp2(cost[c] - ref) - std::exp2(cost[p] - ref) +
                          std::exp2(cc - ref) + std::exp2(cp - ref);
        // space term with size[c] replaced by sz
        const int64_t ko = key(size[c]), kn = key(sz);
        double scn;
        {
            auto top = sizes.rbegin();
            if (kn >= top->first) scn = sz;
            else if (ko == top->first && top->second == 1) {
                auto nx = std::next(top);
                int64_t k2 = nx == sizes.rend() ? kn : std::max(kn, nx->first);
                scn = (double)k2 / 1048576.0;
            } else scn = (double)top->first / 1048576.0;
        }
        const double fn = obj(Sn, scn);
        if (!(fn <= fcur || U01(rng) < std::exp(-beta * (fn - fcur)))) continue;
        // accept: c = (x, z), p = (c, y)
        T.ch0[c] = x;
        T.ch1[c] = z;
        T.par[z] = c;
        if (side) T.ch0[p] = y;
        else T.ch1[p] = y;
        T.par[y] = p;
        std::copy(nu.begin(), nu.end(), T.U.begin() + (size_t)c * W);
        std::copy(no.begin(), no.end(), T.O.begin() + (size_t)c * W);
        std::copy(nlc.begin(), nlc.end(), Lb.begin() + (size_t)c * W);
        if (--sizes[ko] == 0) sizes.erase(ko);
        sizes[kn]++;
        size[c] = sz;
        cost[c] = cc;
        cost[p] = cp;
        S = Sn;
        if (++since >= 4096 || !(S > 1e-200)) {
            resum();
            since = 0;
        }
        fcur = obj(S, sc_now());
        if (fcur < fbest - 1e-12) {
            fbest = fcur;
            b0 = T.ch0;
            b1 = T.ch1;
        }
    }
    return sa_renumber(nl, b0, b1);
}

Tree optimize_tree(const Net &net, int method, int restarts, uint64_t seed) {
    if (method == 0) return greedy_tree(net);
    if (method == 4) {
        // the better of method 1's tree and the bisection tree, then
        // `restarts` rounds of incremental annealing (2000 rotations per
        // leaf each), each from the best tree so far
        Tree best = optimize_tree(net, 1, std::max(2, restarts), seed);
        Plan pb;
        if (!build_plan(net, best, pb).empty()) return best;
        {
            Tree tp = partition_tree(net, std::max(4, restarts), seed);
            Plan pp;
            if (build_plan(net, tp, pp).empty() &&
                (pp.sc_log2 < pb.sc_log2 - 1e-9 ||
                 (std::fabs(pp.sc_log2 - pb.sc_log2) < 1e-9 && pp.tc_log2 < pb.tc_log2))) {
                best = tp;
                pb = pp;
            }
        }
        double bsc = pb.sc_log2, btc = pb.tc_log2;
        const int64_t iters = 2000LL * (int64_t)net.leaf.size();
        for (int r = 0; r < std::max(1, restarts); ++r) {
            Tree t = anneal_tree_fast(net, best, iters, seed + 7919 * (r + 1), bsc - 1.0);
            Plan p;
            if (!build_plan(net, t, p).empty()) continue;
            if (p.sc_log2 < bsc - 1e-9 || (std::fabs(p.sc_log2 - bsc) < 1e-9 && p.tc_log2 < btc)) {
                best = t;
                bsc = p.sc_log2;
                btc = p.tc_log2;
            }
        }
        return best;
    }
    if (method == 2 || method == 3) {
        // anneal from the best heuristic tree (method 2: elimination orders,
        // method 3: recursive bisection), restarts x 20000 rotations, first
        // towards the smallest space complexity seen, then time
        Tree t0 = optimize_tree(net, 1, std::max(2, restarts), seed);
        if (method == 3) {
            // the bisection tree when it beats the elimination heuristics
            Tree tp = partition_tree(net, std::max(4, restarts), seed);
            Plan pe, pp;
            if (build_plan(net, tp, pp).empty() && build_plan(net, t0, pe).empty() &&
                (pp.sc_log2 < pe.sc_log2 - 1e-9 ||
                 (std::fabs(pp.sc_log2 - pe.sc_log2) < 1e-9 && pp.tc_log2 < pe.tc_log2)))
                t0 = tp;
        }
        Plan p0;
        build_plan(net, t0, p0);
        Tree best = t0;
        double bsc = p0.sc_log2, btc = p0.tc_log2;
        for (int r = 0; r < std::max(1, restarts); ++r) {
            Tree t = anneal_tree(net, best, 20000, seed + 7919 * (r + 1), bsc - 1.0);
            Plan p;
            if (!build_plan(net, t, p).empty()) continue;
            if (p.sc_log2 < bsc - 1e-9 || (std::fabs(p.sc_log2 - bsc) < 1e-9 && p.tc_log2 < btc)) {
                best = t;
                bsc = p.sc_log2;
                btc = p.tc_log2;
            }
        }
        return best;
    }
    std::mt19937_64 rng(seed);
    Tree best;
    double bsc = 1e300, btc = 1e300;
    if (restarts < 1) restarts = 1;
    for (int r = 0; r < restarts; ++r) {
        std::vector<int> order = heuristic_order(net, (r % 2) == 0, rng);
        Tree t = tree_from_elimination(net, order);
        Plan p;
        if (!build_plan(net, t, p).empty()) continue;
        if (p.sc_log2 < bsc - 1e-9 || (std::fabs(p.sc_log2 - bsc) < 1e-9 && p.tc_log2 < btc)) {
            bsc = p.sc_log2;
            btc = p.tc_log2;
            best = t;
        }
    }
    Tree g = greedy_tree(net);
    Plan pg;
    if (build_plan(net, g, pg).empty() &&
        (pg.sc_log2 < bsc - 1e-9 || (std::fabs(pg.sc_log2 - bsc) < 1e-9 && pg.tc_log2 < btc)))
        best = g;
    return best;
}

}  // namespace tn

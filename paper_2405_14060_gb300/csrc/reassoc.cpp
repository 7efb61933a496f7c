// Re-association of absorption chains in a contraction tree.
//
// Any binary tree over the same tensors gives the same contraction (Sec.
// "Tensor networks": con is associative; the tree only sets the cost).  Trees
// found by greedy or elimination orders grow a few large tensors by absorbing
// small tensors one at a time (caterpillar chains):
//     Y1 = con(X, W1), Y2 = con(Y1, W2), ..., Yk = con(Y(k-1), Wk).
// Each step reads and writes a large tensor.  Re-associating a run of them as
//     V2 = con(W1, W2), ..., Vk = con(V(k-1), Wk), Yk = con(X, Vk)
// contracts the small tensors among themselves first and streams the large
// tensor once, so the read-write complexity of the run drops by about k while
// the multiply-add count changes by the ratio of the combined small tensor's
// summed x new entries to the single steps' ones.  Runs are chosen per chain
// by dynamic programming over a time model (bytes / bandwidth + FLOPs / rate
// + a fixed cost per launch), under the limits of the streaming kernel (at
// most 32 summed and 32 new combinations per position, 256 together) and a
// bound on the small tensors' size.
#include <algorithm>
#include <cmath>
#include <set>

#include "tn_internal.h"

namespace tn {

namespace {

constexpr double kBW = 4.0e12;        // effective streaming bandwidth, bytes / s
constexpr double kFL = 15.0e12;       // effective streaming FLOP rate
constexpr double kLaunch = 3.0e-6;    // fixed cost of one large-tensor step
constexpr double kSmall = 1.0e-6;     // cost of one small-tensor step
constexpr double kBigMin = 4096;      // a chain's large tensor: at least this many entries
constexpr double kSmallMax = 1024;    // a chain's small tensor: at most this many entries
constexpr double kVMax = 4096;        // combined small tensors: at most this many entries

int pow2ceil(double v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

struct SegCost {
    bool ok = false;
    double t = 0;
};

}  // namespace

Tree reassociate_chains(const Net &net, const Tree &tree) {
    Plan p;
    if (!build_plan(net, tree, p).empty()) return tree;
    const int n = tree.nleaves, NN = 2 * n - 1;
    if (n < 3) return tree;
    auto entries = [&](const std::set<int> &s) {
        double e = 1;
        for (int v : s) e *= net.card[v];
        return e;
    };
    std::vector<std::set<int>> lab(NN);
    for (int id = 0; id < NN; ++id) lab[id] = std::set<int>(p.node[id].labels.begin(),
                                                             p.node[id].labels.end());
    // chain steps: a large operand absorbing a small one
    std::vector<char> step(NN, 0);
    for (int id = n; id < NN; ++id) {
        const Node &nd = p.node[id];
        step[id] = (double)p.node[nd.a].size >= kBigMin && (double)p.node[nd.b].size <= kSmallMax;
    }
    std::vector<int> L(tree.left.begin(), tree.left.end()), R(tree.right.begin(), tree.right.end());
    auto cost = [&](const std::vector<int> &seg, int s, int e) {
        SegCost c;
        const std::set<int> &X = lab[p.node[seg[s]].a], &Y = lab[seg[e - 1]];
        if (e - s == 1) {
            const Node &nd = p.node[seg[s]];
            std::set<int> u = X;
            u.insert(lab[nd.b].begin(), lab[nd.b].end());
            double by = 4 * ((double)p.node[nd.a].size + (double)p.node[nd.b].size + (double)nd.size);
            c.ok = true;
            c.t = by / kBW + 2 * entries(u) / kFL + kLaunch;
            return c;
        }
        // V_i = (W_1 .. W_i) kept where they meet X, Y or a later W
        std::set<int> V;
        for (int i = s; i < e; ++i) {
            const std::set<int> &W = lab[p.node[seg[i]].b];
            V.insert(W.begin(), W.end());
            std::set<int> outside = X;
            outside.insert(Y.begin(), Y.end());
            for (int j = i + 1; j < e; ++j) {
                const std::set<int> &Wj = lab[p.node[seg[j]].b];
                outside.insert(Wj.begin(), Wj.end());
            }
            std::set<int> kept;
            for (int v : V)
                if (outside.count(v)) kept.insert(v);
            V.swap(kept);
            if (entries(V) > kVMax) return c;
        }
        std::set<int> S, T, U = X;
        for (int v : X)
            if (!Y.count(v)) S.insert(v);
        for (int v : Y)
            if (!X.count(v)) T.insert(v);
        U.insert(V.begin(), V.end());
        int ns = pow2ceil(entries(S)), nt = pow2ceil(entries(T));
        if (ns > 32 || nt > 32 || ns * nt > 256) return c;
        double by = 4 * (entries(X) + entries(V) + entries(Y));
        c.ok = true;
        c.t = by / kBW + 2 * entries(U) / kFL + kLaunch + (e - s - 1) * kSmall;
        return c;
    };
    bool changed = false;
    for (int top = n; top < NN; ++top) {
        if (!step[top]) continue;
        int par = p.node[top].parent;
        if (par >= 0 && step[par] && p.node[par].a == top) continue;   // not a chain top
        std::vector<int> seg;   // bottom-up
        for (int c = top;; c = p.node[c].a) {
            seg.push_back(c);
            int a = p.node[c].a;
            if (a < n || !step[a]) break;
        }
        std::reverse(seg.begin(), seg.end());
        const int m = (int)seg.size();
        if (m < 2) continue;
        std::vector<double> dp(m + 1, 1e300);
        std::vector<int> from(m + 1, 0);
        dp[0] = 0;
        for (int e = 1; e <= m; ++e)
            for (int s = e - 1; s >= 0; --s) {
                SegCost c = cost(seg, s, e);
                if (!c.ok) break;   // longer runs only grow the combined tensor
                if (dp[s] + c.t < dp[e]) {
                    dp[e] = dp[s] + c.t;
                    from[e] = s;
                }
            }
        for (int e = m; e > 0; e = from[e]) {
            int s = from[e];
            if (e - s < 2) continue;
            // seg[s .. e-1] = c_1 .. c_k: c_1 <- (W1, W2), c_i <- (c_(i-1), W(i+1)),
            // c_k <- (X, c_(k-1))
            const int k = e - s;
            std::vector<int> c(seg.begin() + s, seg.begin() + e), W(k);
            for (int i = 0; i < k; ++i) W[i] = p.node[c[i]].b;
            const int X = p.node[c[0]].a;
            L[c[0] - n] = W[0];
            R[c[0] - n] = W[1];
            for (int i = 1; i + 1 < k; ++i) {
                L[c[i] - n] = c[i - 1];
                R[c[i] - n] = W[i + 1];
            }
            L[c[k - 1] - n] = X;
            R[c[k - 1] - n] = c[k - 2];
            changed = true;
        }
    }
    if (!changed) return tree;
    // renumber internal nodes in post-order (children before parents; the
    // child holding the earlier original node first, so the original order of
    // independent subtrees is kept)
    Tree out;
    out.nleaves = n;
    std::vector<int> newid(NN, -1);
    for (int id = 0; id < n; ++id) newid[id] = id;
    std::vector<std::pair<int, int>> stack{{NN - 1, 0}};
    while (!stack.empty()) {
        auto &[id, st] = stack.back();
        if (id < n) {
            stack.pop_back();
            continue;
        }
        int a = L[id - n], b = R[id - n];
        if (a > b) std::swap(a, b);
        if (st == 0) {
            st = 1;
            stack.push_back({a, 0});
        } else if (st == 1) {
            st = 2;
            stack.push_back({b, 0});
        } else {
            int me = n + (int)out.left.size();
            out.left.push_back(newid[L[id - n]]);
            out.right.push_back(newid[R[id - n]]);
            newid[id] = me;
            stack.pop_back();
        }
    }
    if (!validate_tree(out).empty() || (int)out.left.size() != n - 1) return tree;
    return out;
}

}  // namespace tn

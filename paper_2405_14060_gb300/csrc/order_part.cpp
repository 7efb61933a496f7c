// Contraction trees by recursive bisection of the tensor network.
//
// The network is read as a hypergraph: one vertex per tensor, one hyperedge
// per label (weight log2 of its domain size) joining the tensors that hold
// it.  Splitting a set of tensors into two halves that share few labels keeps
// the two partial contractions -- and the tensor that joins them -- small, so
// bisecting recursively down to single tensors gives a contraction tree whose
// space complexity follows the cuts (Sec. "Tensor networks": the tree only
// sets the cost; the paper's orders come from such partition-based finders).
// Each bisection is a Fiduccia-Mattheyses local search (move the vertex of
// largest gain, lock it, keep the best balanced prefix) from several random
// balanced starts.
#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>
#include <random>

#include "tn_internal.h"

namespace tn {

namespace {

struct Hyper {
    std::vector<std::vector<int>> vlab;   // labels of each tensor
    std::vector<std::vector<int>> pins;   // tensors of each label
    std::vector<double> w;                // label weight (log2 domain size)
};

// Cut weight of a two-colouring `side` (0/1) of the vertices in S; leaves
// the per-label counts of each side in ca / cb.
double cut_of(const Hyper &H, const std::vector<int> &S, const std::vector<char> &side,
              std::vector<int> &ca, std::vector<int> &cb) {
    std::vector<int> labs;
    for (int x : S)
        for (int v : H.vlab[x]) {
            if (ca[v] == 0 && cb[v] == 0) labs.push_back(v);
            (side[x] ? cb[v] : ca[v])++;
        }
    double cut = 0;
    for (int v : labs)
        if (ca[v] > 0 && cb[v] > 0) cut += H.w[v];
    return cut;
}

// One bisection of S (|S| >= 3) by FM passes from `starts` random balanced
// colourings; returns side[] for the vertices of S.
void bisect(const Hyper &H, const std::vector<int> &S, int starts, std::mt19937_64 &rng,
            std::vector<char> &best_side) {
    const int n = (int)S.size();
    const int lo = std::max(1, (int)std::floor(0.35 * n)), hi = n - lo;   // size of side 1
    std::vector<int> ca(H.pins.size(), 0), cb(H.pins.size(), 0);
    std::vector<char> side(best_side.size(), 0);
    double best = 1e300;
    for (int r = 0; r < starts; ++r) {
        std::vector<int> perm(S);
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int i = 0; i < n; ++i) side[perm[i]] = i < n / 2 ? 1 : 0;
        for (int x : S)
            for (int v : H.vlab[x]) ca[v] = cb[v] = 0;
        double cut = cut_of(H, S, side, ca, cb);
        int n1 = n / 2;
        for (int pass = 0; pass < 8; ++pass) {
            std::vector<char> locked(side.size(), 0);
            std::vector<int> moved;
            double cur = cut, bestp = cut;
            int bestk = 0, cur1 = n1, best1 = n1;
            for (int step = 0; step < n; ++step) {
                // best unlocked move that keeps the sides within bounds
                int bx = -1;
                double bg = -1e300;
                for (int x : S) {
                    if (locked[x]) continue;
                    int to = 1 - side[x];
                    int new1 = cur1 + (to == 1 ? 1 : -1);
                    if (new1 < lo || new1 > hi) continue;
                    double g = 0;
                    for (int v : H.vlab[x]) {
                        int &from_c = side[x] ? cb[v] : ca[v];
                        int &to_c = side[x] ? ca[v] : cb[v];
                        if (from_c == 1 && to_c > 0) g += H.w[v];   // label leaves the cut
                        if (to_c == 0 && from_c > 1) g -= H.w[v];   // label enters the cut
                    }
                    if (g > bg) {
                        bg = g;
                        bx = x;
                    }
                }
                if (bx < 0) break;
                for (int v : H.vlab[bx]) {
                    if (side[bx]) {
                        cb[v]--;
                        ca[v]++;
                    } else {
                        ca[v]--;
                        cb[v]++;
                    }
                }
                cur1 += side[bx] ? -1 : 1;
                side[bx] = 1 - side[bx];
                locked[bx] = 1;
                moved.push_back(bx);
                cur -= bg;
                if (cur < bestp - 1e-12) {
                    bestp = cur;
                    bestk = (int)moved.size();
                    best1 = cur1;
                }
            }
            // roll back the moves after the best prefix
            for (int i = (int)moved.size() - 1; i >= bestk; --i) {
                int x = moved[i];
                for (int v : H.vlab[x]) {
                    if (side[x]) {
                        cb[v]--;
                        ca[v]++;
                    } else {
                        ca[v]--;
                        cb[v]++;
                    }
                }
                side[x] = 1 - side[x];
            }
            n1 = best1;
            if (bestp >= cut - 1e-12) break;
            cut = bestp;
        }
        if (cut < best) {
            best = cut;
            for (int x : S) best_side[x] = side[x];
        }
    }
}

}  // namespace

Tree partition_tree(const Net &net, int starts, uint64_t seed) {
    const int n = (int)net.leaf.size();
    Hyper H;
    H.vlab.resize(n);
    H.pins.resize(net.card.size());
    H.w.resize(net.card.size());
    for (size_t v = 0; v < net.card.size(); ++v) H.w[v] = std::log2((double)std::max(1, net.card[v]));
    for (int x = 0; x < n; ++x)
        for (int v : net.leaf[x]) {
            H.vlab[x].push_back(v);
            H.pins[v].push_back(x);
        }
    Tree t;
    t.nleaves = n;
    if (n < 2) return t;
    std::mt19937_64 rng(seed);
    std::vector<char> side(n, 0);
    std::function<int(std::vector<int>)> build = [&](std::vector<int> S) -> int {
        if (S.size() == 1) return S[0];
        if (S.size() == 2) {
            t.left.push_back(S[0]);
            t.right.push_back(S[1]);
            return n + (int)t.left.size() - 1;
        }
        bisect(H, S, std::max(1, starts), rng, side);
        std::vector<int> A, B;
        for (int x : S) (side[x] ? B : A).push_back(x);
        if (A.empty() || B.empty()) {   // cannot happen with the balance bounds
            A.assign(S.begin(), S.begin() + S.size() / 2);
            B.assign(S.begin() + S.size() / 2, S.end());
        }
        int a = build(A), b = build(B);
        t.left.push_back(a);
        t.right.push_back(b);
        return n + (int)t.left.size() - 1;
    };
    std::vector<int> all(n);
    std::iota(all.begin(), all.end(), 0);
    build(all);
    return t;
}

}  // namespace tn

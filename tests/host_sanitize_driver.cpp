// Host-side driver for the address / undefined-behaviour sanitizer check of
// libtn's planner and model I/O (tests/test_host_sanitizers_cpu.py builds it
// with -fsanitize=address,undefined together with csrc/plan.cpp,
// csrc/order_part.cpp, csrc/reassoc.cpp and csrc/model.cpp).  It runs every
// order-search method, tree validation, planning and chain re-association on
// small networks of each structure class, and the UAI parser on valid and
// malformed files; any sanitizer report aborts with a non-zero status.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <random>
#include <string>
#include <vector>

#include "model.h"
#include "tn_internal.h"

using namespace tn;

namespace {

int failures = 0;

void check(bool ok, const std::string &what) {
    if (!ok) {
        std::fprintf(stderr, "FAILED: %s\n", what.c_str());
        ++failures;
    }
}

// The model's network as the library builds it: factor leaves, then one
// unity vector per variable (batched: those carry the evidence-batch label).
Net network(const std::vector<int> &card, const std::vector<Labels> &scopes, bool batched) {
    Net n;
    n.card = card;
    for (const auto &s : scopes) {
        n.leaf.push_back(s);
        n.leaf_beta.push_back(0);
    }
    for (int v = 0; v < (int)card.size(); ++v) {
        n.leaf.push_back(Labels{v});
        n.leaf_beta.push_back(batched ? 1 : 0);
    }
    return n;
}

Net grid(int L, bool batched) {
    std::vector<int> card(L * L, 2);
    std::vector<Labels> sc;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            if (j + 1 < L) sc.push_back({i * L + j, i * L + j + 1});
            if (i + 1 < L) sc.push_back({i * L + j, (i + 1) * L + j});
            sc.push_back({i * L + j});
        }
    return network(card, sc, batched);
}

// Random 3-regular multigraph by pairing, loops dropped.
Net regular3(int n, uint64_t seed) {
    std::mt19937_64 rng(seed);
    std::vector<int> stubs;
    for (int v = 0; v < n; ++v)
        for (int k = 0; k < 3; ++k) stubs.push_back(v);
    std::shuffle(stubs.begin(), stubs.end(), rng);
    std::vector<Labels> sc;
    for (size_t i = 0; i + 1 < stubs.size(); i += 2)
        if (stubs[i] != stubs[i + 1]) sc.push_back({stubs[i], stubs[i + 1]});
    return network(std::vector<int>(n, 2), sc, false);
}

// Banded random DAG with domain sizes 2..4 (Bayesian-network structure).
Net bayes(int n, uint64_t seed) {
    std::mt19937_64 rng(seed);
    std::vector<int> card(n);
    for (auto &c : card) c = 2 + (int)(rng() % 3);
    std::vector<Labels> sc;
    for (int v = 0; v < n; ++v) {
        Labels s;
        int np = (int)(rng() % 4);
        for (int k = 0; k < np && v - 1 - k >= 0; ++k) s.push_back(v - 1 - (int)(rng() % std::min(v, 4)));
        std::sort(s.begin(), s.end());
        s.erase(std::unique(s.begin(), s.end()), s.end());
        s.push_back(v);
        sc.push_back(s);
    }
    return network(card, sc, false);
}

void exercise(const std::string &name, const Net &net) {
    for (int method = 0; method <= 4; ++method) {
        Tree t = optimize_tree(net, method, 2, 7 + method);
        check(validate_tree(t).empty(), name + ": method " + std::to_string(method) + " tree");
        Plan p;
        check(build_plan(net, t, p).empty(), name + ": plan of method " + std::to_string(method));
        check(build_plan(net, t, p, 64).empty(), name + ": GEMM-form plan");
        Tree r = reassociate_chains(net, t);
        Plan pr;
        check(validate_tree(r).empty() && build_plan(net, r, pr).empty(),
              name + ": re-associated tree of method " + std::to_string(method));
    }
    std::vector<int> order(net.card.size());
    for (int v = 0; v < (int)order.size(); ++v) order[v] = (int)order.size() - 1 - v;
    Tree te = tree_from_elimination(net, order);
    check(validate_tree(te).empty(), name + ": elimination tree");
    Tree tp = partition_tree(net, 3, 5);
    check(validate_tree(tp).empty(), name + ": bisection tree");
    Tree ta = anneal_tree(net, te, 500, 3, 10.0);
    check(validate_tree(ta).empty(), name + ": annealed tree");
    Tree tf = anneal_tree_fast(net, te, 20000, 3, 10.0);
    check(validate_tree(tf).empty(), name + ": incrementally annealed tree");
    // malformed trees are rejected, not read out of bounds
    Tree bad = te;
    if (!bad.left.empty()) {
        bad.left[0] = bad.right[0];
        check(!validate_tree(bad).empty(), name + ": repeated child rejected");
        bad = te;
        bad.left.back() = 10 * bad.nleaves;
        check(!validate_tree(bad).empty(), name + ": out-of-range child rejected");
    }
}

void uai_cases(const std::string &dir) {
    const std::string good = dir + "/good.uai", trunc = dir + "/trunc.uai", neg = dir + "/neg.uai";
    {
        std::ofstream f(good);
        f << "MARKOV\n3\n2 3 2\n2\n2 0 1\n2 1 2\n\n6\n1 2 3 4 5 6\n\n6\n0.5 1 1.5 2 2.5 3\n";
    }
    {
        std::ofstream f(trunc);
        f << "MARKOV\n3\n2 3 2\n2\n2 0 1\n2 1 2\n\n6\n1 2 3\n";
    }
    {
        std::ofstream f(neg);
        f << "BAYES\n1\n2\n1\n1 0\n\n2\n-0.5 1.5\n";
    }
    ModelData m;
    bool perr = false;
    check(model_from_uai(good.c_str(), m, perr).empty() && m.nvars == 3 && m.nfactors == 2,
          "UAI: valid file");
    ModelData m2;
    perr = false;
    check(!model_from_uai(trunc.c_str(), m2, perr).empty(), "UAI: truncated file rejected");
    ModelData m3;
    perr = false;
    check(!model_from_uai(neg.c_str(), m3, perr).empty(), "UAI: negative entry rejected");
    ModelData m4;
    perr = false;
    check(!model_from_uai((dir + "/missing.uai").c_str(), m4, perr).empty(), "UAI: missing file");
    const int card[2] = {2, 0}, off[2] = {0, 2}, vars[2] = {0, 1};
    const double tab[4] = {1, 1, 1, 1};
    ModelData m5;
    check(!model_from_arrays(2, card, 1, off, vars, tab, m5).empty(), "arrays: zero domain rejected");
}

}  // namespace

int main(int argc, char **argv) {
    const std::string dir = argc > 1 ? argv[1] : ".";
    exercise("grid 5x5", grid(5, false));
    exercise("grid 4x4 batched", grid(4, true));
    exercise("3-regular 24", regular3(24, 11));
    exercise("Bayesian network 30", bayes(30, 13));
    uai_cases(dir);
    if (failures) {
        std::fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    std::printf("host sanitizer driver ok\n");
    return 0;
}

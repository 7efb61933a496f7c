// Internal data structures of libtn: tensor networks, contraction trees and
// per-node plans (host side).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "tn.h"

namespace tn {

using Labels = std::vector<int>;

// A tensor network (Lambda, T, V0) (Def. "Tensor Network"): leaf label lists
// in storage order (last label fastest), label sizes, output labels V0.  A
// leaf may also carry the evidence-batch label (always outermost), which is
// kept to the root.
struct Net {
    std::vector<int> card;            // size of every label
    std::vector<Labels> leaf;         // labels of each leaf
    std::vector<char> leaf_beta;      // leaf carries the batch label
    Labels out;                       // V0
};

// Binary contraction tree over nleaves leaves: internal node i has id
// nleaves + i and children left[i], right[i] (Sec. Tensor networks).
struct Tree {
    int nleaves = 0;
    std::vector<int> left, right;
};

// Plan of one tensor of the tree (leaf or internal node).
struct Node {
    Labels labels;        // storage order, batch label excluded
    bool beta = false;    // carries the batch label (outermost dimension)
    int64_t size = 1;     // entries per batch item
    int a = -1, b = -1;   // operands: a is the larger (its layout is kept)
    Labels elim;          // labels summed/maximised here, in kernel K order
    double muladds = 0;   // prod over the union of operand labels (per item)
    int parent = -1;
    int depth = 0;
    // dense GEMM form C[bt, m, n] = sum_k A[bt, m, k] B[bt, k, n], chosen when
    // every group is large and no label is summed inside one operand alone
    bool gemm = false;
    int ga = -1, gb = -1; // operand on the row (m) side, on the column (n) side
    Labels gbt, gm, gn;   // batch, row and column labels (elim holds k)
};

struct Plan {
    Net net;
    Tree tree;
    std::vector<Node> node;           // leaves first, then internal nodes
    int root = -1;
    double tc_log2 = 0, sc_log2 = 0, rw_log2 = 0;
    double total_muladds = 0, total_rw_entries = 0;
};

std::string validate_tree(const Tree &t);
// gemm_min: a node takes the GEMM form when its m, n and k groups each hold
// at least gemm_min entries per item (0 disables the GEMM form).
std::string build_plan(const Net &net, const Tree &tree, Plan &plan, int64_t gemm_min = 0);
Tree greedy_tree(const Net &net);
Tree tree_from_elimination(const Net &net, const std::vector<int> &order);
Tree optimize_tree(const Net &net, int method, int restarts, uint64_t seed);
// Tree from recursive bisection of the tensor hypergraph (order_part.cpp).
Tree partition_tree(const Net &net, int starts, uint64_t seed);
// Equivalent tree with runs of absorption steps re-associated (reassoc.cpp).
Tree reassociate_chains(const Net &net, const Tree &tree);
Tree anneal_tree(const Net &net, const Tree &start, int iters, uint64_t seed, double sc_target);
// The same annealing, evaluated incrementally (a move updates one node).
Tree anneal_tree_fast(const Net &net, const Tree &start, int64_t iters, uint64_t seed,
                      double sc_target);
double log2_size(const Net &net, const Labels &l);

}  // namespace tn

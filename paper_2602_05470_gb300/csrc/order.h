// Contraction trees, their cost model, the order finder and dynamic slicing.
//
// Cost model (paper: the paragraph after the MWIS construction): time complexity
// = total multiply-adds, here sum over internal nodes of 2^{|labels of both
// children|}; space complexity = the largest intermediate tensor, 2^{max |labels|}.
// Eq. (4): rho = sum over tensors of max(0, log2|T| - log2 T_target).
#pragma once
#include <stdint.h>

#include <vector>

namespace bbtn {

struct CNode {
    int l = -1, r = -1, parent = -1;
    int leaf = -1;               // index of the network tensor (leaves only)
    std::vector<int> lab;        // output labels, ascending
    bool is_leaf() const { return l < 0; }
};

struct CTree {
    std::vector<CNode> nodes;    // leaves first (node i = tensor i), then internal nodes
    int root = -1;
    int nleaves = 0;
};

struct Cost {
    double tc_log2 = 0;          // log2 of sum of 2^{|union|} over internal nodes
    int sc = 0;                  // max label count over all nodes
    double rho = 0;              // Eq. (4) with T_target = 2^cap
};

// Labels of internal nodes recomputed from the leaves' labels (a label stays while
// some leaf outside the subtree still carries it).
void recompute_labels(CTree &t);

// Cost of the tree when the variables with removed[v] != 0 are fixed.
Cost tree_cost(const CTree &t, int cap, const std::vector<char> *removed = nullptr);

// Greedy pairwise order: repeatedly contract the pair of tensors sharing a label
// that minimises 2^{|out|} - 2^{|A|} - 2^{|B|}; `noise` > 0 randomises ties.
CTree greedy_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, uint64_t seed,
                   double noise);

// Contraction tree from a min-fill variable elimination order (bucket elimination:
// the tensors holding the next variable are contracted together, smallest first).
CTree elimination_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, uint64_t seed);

struct SAParams {
    double beta_start = 1.0, beta_end = 15.0;
    int beta_steps = 20;
    int sweeps = 1;              // moves per beta step = sweeps * internal nodes
    int cap = 30;                // T_target exponent for rho
    double w_rho = 1.0;          // weight of rho in the objective
};

// Simulated annealing over subtree rotations ((a,b),y) -> ((a,y),b) minimising
// log2(tc) + w_rho * rho.
void tree_sa(CTree &t, const SAParams &sp, uint64_t seed);

// Greedy + annealing with several restarts; returns the best tree. Restart 1 starts
// from a min-fill elimination order, the others from greedy orders; with
// minfill_odd every odd restart starts from a min-fill order (each with its own
// tie-breaking seed).
CTree find_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, int cap, double w_rho,
                 int trials, int sa_beta_steps, uint64_t seed, bool minfill_odd = false);

// Dynamic slicing: pick labels to fix (greedily, the one that lowers the
// overflow most, then the one adding least time) until every tensor fits 2^cap.
// Re-anneals the sliced tree in between. Returns the sliced labels; `t` becomes
// the tree of one slice.
std::vector<int> dynamic_slicing(CTree &t, int cap, int sa_beta_steps, uint64_t seed);

}  // namespace bbtn

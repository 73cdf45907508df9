// Problem instances and their tropical tensor networks (paper: Tropical Tensor
// Networks section -- Eq. (1), the edge matrices B^{ij} and vertex vectors w^i,
// and the MWIS construction with the hard constraint).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace bbtn {

enum Kind { kSpin = 0, kMwis = 1 };

struct Problem {
    int kind = kSpin;
    int n = 0;
    std::vector<int> ei, ej;        // edges (ei[k] < ej[k])
    std::vector<int32_t> J;         // spin: couplings
    std::vector<int32_t> h2;        // spin: 2 * field
    std::vector<int32_t> w;         // mwis: weights
    std::vector<std::vector<std::pair<int, int>>> adj;   // (neighbour, edge index)
    int m() const { return (int)ei.size(); }
    bool zero_field() const;
    void build_adjacency();
};

// Validates and normalises (edge endpoints ordered, no self loops / duplicates,
// magnitudes within the int32 value range of the semiring). Throws Error.
void validate(Problem &p);
Problem read_problem_file(const std::string &path);

// A tensor of the network: labels are variable ids (bit i <-> labels[i]); values
// are the max-plus entries (negated energies, x2 for spin glasses); counts are 1
// for finite entries and 0 for the -infinity sentinel.
struct TensorDef {
    std::vector<int> labels;
    std::vector<int32_t> val;
};

// Max-plus network of -2H (spin glass) or of the MWIS weight. Each vertex vector
// is folded into its first incident edge matrix (same network value, fewer
// tensors); isolated vertices keep their own vector.
std::vector<TensorDef> build_network(const Problem &p);

// Objective of a full assignment x (0/1 per variable): -2H for spin glasses
// (s = 2x - 1), the set weight for MWIS (INT64_MIN if not independent).
int64_t objective(const Problem &p, const std::vector<int8_t> &x);

// Objective of the variables already fixed plus a rigorous upper bound on what
// the free part can add (global pruning bound of the branch-and-bound driver).
// fx[v] = -1 (free), 0 or 1.
int64_t upper_bound(const Problem &p, const std::vector<int8_t> &fx);

}  // namespace bbtn

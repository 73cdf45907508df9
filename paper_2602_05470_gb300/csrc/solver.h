// Host-driven solver: plain contraction, dynamic slicing and the branch-and-bound
// tensor network driver (paper: TN with Slicing and Branch-and-Bound Tensor
// Network sections).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/bbtn.h"
#include "exec.h"
#include "gnn.h"
#include "network.h"
#include "order.h"

namespace bbtn {

// Empties the process-wide cache of root contraction orders.
void clear_order_cache();

struct SolveOutput {
    int64_t value = 0;                 // max-plus value of the network (-2H* or alpha)
    std::vector<uint64_t> res;         // one residue per modulus: the CRT ones, then the check plane's
    std::vector<uint64_t> primes;      // the moduli, in the same order
    int n_crt = 0;                     // residues that enter the CRT
    bool checked = false;              // the residues after the first n_crt are the overflow check
    std::vector<int8_t> x;             // optimal configuration (0/1 per variable)
    bool have_x = false;
};

// Per-node records of a dry search (training data of the learned branch scorer).
struct BranchLog {
    int max = 0;              // rows available
    int lookahead = 1;        // candidates the search itself compares
    int count = 0;            // rows written
    std::vector<int8_t> fx;   // max x n fixings
    std::vector<float> score; // max x n overflow score / its maximum
    std::vector<float> gamma; // max x n: gamma of the branching seeded at v (-1: not a candidate, 0: infeasible)
};

class Solver {
  public:
    Solver(const bbtn_opts &o, cudaStream_t s, Arena *arena, TileTuner *tuner = nullptr)
        : opts_(o), stream_(s), arena_(arena), tuner_(tuner) {
        prog_.stream = s;
    }
    ~Solver() {
        try {
            shard_release();
        } catch (...) {
        }
    }
    SolveOutput solve(const Problem &p, bool want_count, bool want_config, bbtn_stats *st);
    // host-only planning summary (bbtn_analyze)
    void analyze(const Problem &p, bbtn_plan_info *info, const char *dump_path);
    // learned scorers (used with opts.use_gnn; borrowed): `branch` picks the seed of
    // each branching region, `value` predicts an optimum (first incumbent and the
    // order of children, MWIS only)
    void set_gnn(GnnModel *branch, GnnModel *value) {
        gnn_branch_ = branch;
        gnn_ = value;
    }
    // dry search of the loaded problem with per-node lookahead records (host only)
    void branch_samples(const Problem &p, BranchLog *log, bbtn_stats *st);
    // host-only set-up: instance network and root contraction order (into the order cache)
    void prepare(const Problem &p, bbtn_stats *st);
    // dry search: the fixings of its leaf sub-networks, n per leaf (host only)
    void search_leaves(const Problem &p, int64_t max_leaves, std::vector<int8_t> &fx, bbtn_stats *st);

    // Branch sharding across ranks. Every rank expands the same search tree on the
    // host (the dry search: only the heuristic incumbent prunes, so the leaf list
    // does not depend on the rank) and takes the leaves i = rank (mod world).
    // shard_values contracts them value-only and returns the largest leaf maximum
    // (kNeg if none is feasible); shard_counts, given the maximum over all ranks,
    // contracts with counts this rank's leaves that attain it and returns its part
    // of the counting sum (value kNeg and zero counts if it holds none).
    int64_t shard_values(const Problem &p, int rank, int world, bool want_count, bbtn_stats *st);
    struct ShardResult {
        int32_t value = kNeg;
        std::vector<uint64_t> planes, moduli;   // one word per count plane (pair or wide form)
        int n_crt_planes = 0;
        std::vector<int8_t> x;                  // an optimal configuration, if this rank holds one
        bool have_x = false;
    };
    ShardResult shard_counts(int64_t global_max, bool want_config);
    void shard_release();

  private:
    struct Leafset;
    void setup(const Problem &p, int active_solves, bool want_count);
    void setup_host(const Problem &p, bool want_count);
    std::vector<int32_t> contract_leaves(const std::vector<std::vector<int8_t>> &leaves, bool counting = true,
                                         const CTree *tree = nullptr);
    void window_open();
    void enqueue_leaves(const std::vector<std::vector<int8_t>> &leaves, bool counting, const CTree *tree, int64_t s0);
    std::vector<int32_t> window_close(int64_t n, bool aggregate);
    void note_leaf_values(const std::vector<std::vector<int8_t>> &leaves, const std::vector<int32_t> &vals);
    struct Window {
        bool open = false;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        double tw = 0;
        RunStats rs;
    };
    Window win_;
    std::vector<int8_t> *leaf_log_ = nullptr;   // search_leaves: leaf fixings
    int64_t leaf_log_max_ = 0;
    bool leaf_order(const std::vector<int8_t> &fx, CTree &out);
    void finish(bool want_config);
    void run_plain();
    void run_sliced();
    void run_bbtn();
    void search(bool dry, BranchLog *log);
    int64_t incumbent_heuristic();
    int64_t incumbent_learned();
    void simplify(std::vector<int8_t> &fx) const;
    CTree order_for(const std::vector<int8_t> &fx, int cap, double w_rho, int trials, bool minfill_odd = false);
    CTree cached_order(const std::vector<int8_t> &fx, int cap, double w_rho, int trials, bool minfill_odd = false);

    bbtn_opts opts_;
    cudaStream_t stream_;
    Arena *arena_;
    const Problem *p_ = nullptr;
    DeviceNetwork net_;
    CTree tree_;                        // reference tree (labels of the free network)
    std::vector<int8_t> fx0_;           // root fixed variables (symmetry)
    int np_ = 0, n_crt_ = 0;
    bool pair_ = true;                  // count planes hold two residues mod 30-bit primes
    bool check_ = false;
    std::vector<uint64_t> primes_;
    uint32_t cprime_[kMaxPlanes] = {0};
    uint64_t mult_ = 1;                 // count multiplier from symmetry
    // device accumulator of branch results: slot 0 = running counting-sum
    int32_t *d_val_ = nullptr;
    uint64_t *d_cnt_ = nullptr;
    int64_t dcap_ = 0;
    uint64_t arena_budget_ = 1ull << 30;   // bytes the leaf arenas of one launch group may use
    void *d_scratch_ = nullptr;
    size_t scratch_bytes_ = 0;
    // best leaf (for the configuration)
    int64_t best_val_ = INT64_MIN;
    std::vector<int8_t> best_fx_;
    int64_t incumbent_ = INT64_MIN;
    bbtn_stats *st_ = nullptr;
    SolveOutput out_;
    Profiler prof_;
    TileTuner *tuner_ = nullptr;        // borrowed from the context (kept across solves)
    DeviceBuf prog_;                    // fused-subtree programs
    GnnModel *gnn_ = nullptr;
    GnnModel *gnn_branch_ = nullptr;
    std::vector<float> logit_;          // model logits of x_v = 1 at the root
    void ensure_buffers(int64_t n);
    void release_buffers();
    // branch sharding state (between shard_values and shard_counts)
    std::vector<std::vector<int8_t>> shard_leaves_;
    std::vector<int32_t> shard_vals_;
    bool shard_open_ = false;
};

}  // namespace bbtn

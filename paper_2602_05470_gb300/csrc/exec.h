// Contraction executor: turns (network, tree, fixed variables) into a list of
// device steps with a static arena layout, runs them on a stream, and walks the
// tree backwards to recover an optimal configuration.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "network.h"
#include "order.h"

namespace bbtn {

// The network's original tensors, resident on the device for the whole solve.
struct DeviceNetwork {
    int nvars = 0;
    int32_t *vals = nullptr;                 // all tensors' values, concatenated
    std::vector<uint64_t> offset;            // element offset of tensor i
    std::vector<std::vector<int>> labels;    // bit i <-> labels[i]
    std::vector<int32_t> host_vals;          // staged values (set_host), uploaded by upload()
    int64_t value_bound = 0;                 // sum over tensors of the largest |finite entry|:
                                             // bounds |value| of every intermediate entry
    void set_host(const std::vector<TensorDef> &ts, int nvars);
    void upload(cudaStream_t s);
    void release(cudaStream_t s = nullptr);   // stream-ordered free
    ~DeviceNetwork() { release(); }
};

// Where an operand of a step lives.
struct Ref {
    int kind = 0;          // 0: network tensor, 1: arena block, 2: external (root destination)
    uint64_t off = 0;      // kind 0: element offset in DeviceNetwork::vals; kind 1: byte offset
    uint64_t plane = 0;    // count-plane stride in elements
    uint64_t base = 0;     // constant element offset (fixed bits)
    int rank = 0;          // kind 1: rank of the block (planes of 2^rank elements)
};

struct PStep {
    ContractParams P;      // pointers filled at launch from the refs
    Ref a, b, c;
    int node = -1;
    int a_node = -1, b_node = -1;   // tree nodes read as operand A / B
    int lab_c[32];         // output labels (bit order of C)
    double ops = 0;        // 2^{|union|} multiply-adds
    double bytes = 0;      // algorithmic bytes (operands read once, result written once)
    uint64_t c_block = 0;  // arena bytes of the result (kind 1)
    bool fused = false;    // runs inside a fused small-subtree block
    std::vector<int> lab_a, lab_b;   // label at each physical bit of A / B (-1: fixed bit)
    // K1m chains (value-only plans): chain_len = L > 0 on the last step of a fused
    // chain (it writes the chain's result), -1 on the chain's earlier steps (their
    // results are never materialised)
    int chain_len = 0;
    int chain_first = -1;  // the chain's first step (on the last step)
    ChainParams chain;     // kernel parameters, pointers filled at launch
    Ref chain_a;           // the chain's A operand
    uint64_t chain_b[kChainMaxSteps] = {0};   // element offsets of the B operands in the network values
};

struct Plan {
    std::vector<PStep> steps;
    size_t arena_bytes = 0;
    int np = 0;
    double ops = 0, bytes = 0;
    int max_rank = 0;
    // per tree node: its step index (internal) and the bit order of its result
    std::vector<int> node_step;
    std::vector<std::vector<int>> node_layout;
    // fused small subtrees (one launch before the remaining steps)
    std::vector<FStep> fsteps;
    std::vector<FSub> fsubs;
    size_t fused_smem = 0;
    int64_t fused_steps = 0;
    // scratch of the split-K steps (K1s), at the end of the arena
    uint64_t splitk_off = 0, splitk_bytes = 0;
    int64_t chains = 0, chained_steps = 0;   // K1m chains and the steps they replace
};


// Element layout of an arena block of rank r with np count planes.
size_t block_bytes(int r, int np);
uint64_t count_plane_offset_bytes(int r);

// Plan the contraction of the network restricted to fx (fx[v] = -1 free, else the
// fixed value). The result (a scalar) goes to the external destination given at
// run time. keep_all keeps every intermediate alive (for the backward walk).
// chains: fuse chains of value-only streaming steps (K1m; plans with np == 0 and
// without keep_all only).
Plan make_plan(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx, int np,
               const uint32_t *cprime, bool keep_all, bool chains = true);

// Per-launch CUDA-event timing of contraction kernels (profile mode): an event
// pair on the launching stream around each launch, read back after a sync.
struct Profiler {
    struct Rec { cudaEvent_t a, b; double bytes, ops; int ra, rb, rc, rs, ident, kind, n; };
    FILE *dump = nullptr;    // optional CSV of every launch (BBTN_PROFILE_DUMP)
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    size_t used = 0;
    double ms = 0, bytes = 0, ops = 0;
    int64_t launches = 0;
    // per kernel; kind: 0 streaming value-only, 1 fused, 2 tiled value-only (int32),
    // 3 split-K, 4 tiled value-only (16-bit lanes), 5 tiled counting, 6 streaming counting,
    // 7 fused chain (K1m)
    double chain_ms = 0, chain_bytes = 0;
    int64_t chain_launches = 0;
    double stream_ms = 0, stream_bytes = 0, scount_ms = 0, scount_bytes = 0;
    double tiled_ms = 0, tiled_ops = 0, tcount_ms = 0, tcount_ops = 0, tiled_bytes = 0, tcount_bytes = 0;
    int64_t stream_launches = 0, scount_launches = 0, tiled_launches = 0, tiled16_launches = 0, tcount_launches = 0;
    cudaEvent_t get();
    void collect();          // after the stream has been synchronised
    ~Profiler();
};

// Autotuner of the tiled kernel's load layout (which operand dimension its lanes
// run along, for A and for B): the first launch of a step signature times all four
// choices on the real step (each writes the same result) and keeps the fastest
// for every later launch with that signature.
struct TileTuner {
    std::unordered_map<uint64_t, int> best;   // signature -> lanes (0..3)
    int64_t tuned = 0;                        // signatures timed so far
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int pick(uint64_t key, const std::function<cudaError_t(int)> &launch, cudaStream_t s);
    ~TileTuner();
};

struct RunStats {
    int64_t launches = 0;
    int64_t chains = 0, chained_steps = 0;
    double ops = 0, bytes = 0;
    Profiler *prof = nullptr;
    TileTuner *tuner = nullptr;
};

// Grow-only device buffer for the fused-subtree programs, allocated and freed in
// the order of `stream` (no device-wide synchronisation, so solves on other
// streams keep running).
struct DeviceBuf {
    void *ptr = nullptr;
    size_t size = 0;
    cudaStream_t stream = nullptr;
    void reserve(size_t bytes);
    ~DeviceBuf();
};

// K1m parameters (pointers excepted) of a chain given by its labels: A's label at
// each physical bit (-1: fixed), and per step the labels of B_l at its physical
// bits and of the step's result. False if the chain does not fit the kernel.
bool chain_params(const std::vector<int> &lab_a, const std::vector<std::vector<int>> &lab_b,
                  const std::vector<std::vector<int>> &lab_c, ChainParams &cp);

// Enqueue a plan: arena = device base pointer of at least plan.arena_bytes,
// root result to (out_val[0], out_cnt[t * out_plane]); prog holds the fused
// program while it runs (stream-ordered reuse across plans).
void run_plan(const Plan &plan, const DeviceNetwork &net, char *arena, int32_t *out_val,
              uint64_t *out_cnt, uint64_t out_plane, cudaStream_t s, RunStats *st, DeviceBuf *prog);

// Enqueue the plans of up to kBatchMax leaf sub-networks of one tree together:
// leaf i uses the arena at arena + i * stride and writes its root result to
// (out_val[i], out_cnt[t * out_plane + i]). The fused subtrees of every leaf run in
// one launch; each remaining tree node runs as one launch per kernel for all
// leaves (paper Eq. (3): the leaves are the sliced sub-networks of one network).
void run_plans(const std::vector<const Plan *> &plans, const DeviceNetwork &net, char *arena, uint64_t stride,
               int32_t *out_val, uint64_t *out_cnt, uint64_t out_plane, cudaStream_t s, RunStats *st,
               DeviceBuf *prog);

// Configuration recovery (the tropical backward pass) within a device-memory
// budget. The forward pass keeps only checkpoint intermediates, chosen so that
// every subtree segment between checkpoints fits a share of the budget; the walk
// then goes top-down in an order fixed by the tree alone, recomputes a missing
// child's segment just before the walk needs it, and releases each tensor after
// its own backward step. Selections stay on the device (one int64 slot per tree
// node, read and written by the backward kernels), so the whole walk is enqueued
// without waiting and read back once.
struct BwdAction {
    int kind = 0;          // 0: recompute the step of `node`, 1: backward of `node`
    int node = -1;
    Ref a, b, c;           // operands and result, arena offsets resolved
};
struct BackwardPlan {
    Plan fwd;              // values-only forward that keeps the checkpoints
    std::vector<BwdAction> actions;
    size_t arena_bytes = 0;          // forward and walk peak + selections + split-K scratch
    uint64_t sel_off = 0;            // byte offset of the selection array (nodes + 1 int64)
    uint64_t scratch_off = 0, scratch_bytes = 0;
    int64_t kept = 0, recomputed = 0;
    double peak_bytes = 0;           // tensor bytes alive at most (forward and walk)
    double keep_all_bytes = 0;       // what keeping every intermediate takes
};
BackwardPlan make_backward_plan(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx,
                                uint64_t budget);
// Runs the forward (root value to root_val) and the walk; sets x[v] for every free
// variable (fixed ones copied from fx). One synchronisation of the stream, at the end.
void run_backward(const BackwardPlan &bp, const CTree &t, const DeviceNetwork &net, char *arena,
                  int32_t *root_val, const std::vector<int8_t> &fx, std::vector<int8_t> &x, cudaStream_t s,
                  RunStats *st, DeviceBuf *prog);

// Grow-only device arena, allocated and freed in the order of `stream` (the owning
// solver's), so growing it does not wait for other contexts' work on the device.
struct Arena {
    char *ptr = nullptr;
    size_t size = 0;
    bool owned = true;
    cudaStream_t stream = nullptr;
    void reserve(size_t bytes);
    void adopt(void *p, size_t bytes);       // caller-owned workspace
    void release();
    ~Arena() { release(); }
};

}  // namespace bbtn

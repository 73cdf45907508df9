// Internal (C++) interface between the host planner and the sm_103a kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "semiring.cuh"

namespace bbtn {

// The largest dynamic shared memory a kernel may be launched with is a property of
// the function on each device (cudaFuncSetAttribute), shared by every host thread
// of the process. Each kernel that takes more than 48 KB gets it once per device,
// at the device's opt-in maximum less its static shared memory, so that launches of
// different sizes from concurrent host threads (several contexts, one per stream)
// never race on it.
template <auto Kernel>
cudaError_t allow_max_dynamic_smem() {
    constexpr int kMaxDevices = 64;
    static std::once_flag once[kMaxDevices];
    static cudaError_t err[kMaxDevices];
    int dev = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r != cudaSuccess) return r;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        int optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, Kernel);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        err[dev] = e;
    });
    return err[dev];
}

// One operand of a pairwise step. Element e of the operand lives at
// val[base + e] and cnt[t * plane + base + e]; `base` carries the constant
// offset of variables fixed by slicing / branching (paper Eq. (3): the reduced
// network T|_{s_Vf = x} reads a sub-block of each original tensor).
struct Operand {
    const int32_t *val = nullptr;
    const uint64_t *cnt = nullptr;
    uint64_t plane = 0;       // elements between count planes
    uint64_t base = 0;        // constant element offset
    int unit_counts = 0;      // 1: counts implied by values (1 if finite, else 0)
};

// C[o] = max(NEG, max_k A[offA(o) + kA(k)] + B[offB(o) + kB(k)]) with counts.
// Output bit i of o sits at bit oA[i] of A's index (-1: not in A), likewise oB;
// summed bit j of k sits at bit sA[j] / sB[j].
struct ContractParams {
    Operand A, B;
    int32_t *vc = nullptr;
    uint64_t *cc = nullptr;
    uint64_t planeC = 0;
    int rc = 0, rs = 0, hasB = 0, np = 0;
    int8_t oA[32], oB[32], sA[32], sB[32];
    uint32_t cprime[kMaxPlanes];
    // value-only steps: 1 if every finite value of both operands and of the result
    // is known to lie in (-2^13, 2^13) -- the tiled kernel then adds and maxes two
    // 16-bit values per instruction (int32 in memory, infeasible results as NEG)
    int v16 = 0;
};

// Picks the kernel: the register-tiled one (K1t) for large two-operand steps, else
// the streaming gather kernel (K1 / K3).
cudaError_t launch_contract(const ContractParams &p, cudaStream_t s, int *kind = nullptr, void *scratch = nullptr,
                            size_t scratch_bytes = 0);   // kind: 0 K1/K3, 2 K1t, 3 K1s
// K1s: split-K for steps with at most 2^kSplitKMaxOutBits outputs (one grid row per
// output) and long sums (splitk_eligible). scratch: device buffer of
// splitk_scratch_bytes(rc, np).
constexpr int kSplitKMaxOutBits = 15;
bool splitk_eligible(const ContractParams &p);
size_t splitk_scratch_bytes(int rc, int np);
cudaError_t launch_contract_splitk(const ContractParams &p, void *scratch, size_t bytes, cudaStream_t s);
// K1t only; cudaErrorNotSupported when the step's shape does not fit it.
cudaError_t launch_contract_tiled(const ContractParams &p, cudaStream_t s);
// K1 / K3 only (four outputs per thread when rc >= 2, else one).
cudaError_t launch_contract_stream(const ContractParams &p, cudaStream_t s);
// K1v: four consecutive outputs per thread; cudaErrorNotSupported when rc < 2.
cudaError_t launch_contract_stream4(const ContractParams &p, cudaStream_t s);
bool stream4_eligible(const ContractParams &p);

// Leaf-batched launches: the same tree node's step of up to kBatchMax leaf
// sub-networks in one launch, each entry with its own operands, output and shape
// (all entries: same np and hasB). cudaErrorNotSupported if an entry does not fit.
constexpr int kBatchMax = 16;
cudaError_t launch_contract_stream4_batch(const ContractParams *p, int n, cudaStream_t s);
// lanes: -1 = lanes along k for an operand whose bit 0 is a summed label, else along
// m / n; 0..3 = forced (bit 0: A along k, bit 1: B along k), as an autotuner picks it
cudaError_t launch_contract_tiled_batch(const ContractParams *p, int n, cudaStream_t s, int lanes = -1);
bool tiled_eligible(const ContractParams &p);
bool tiled_uses_v16(const ContractParams &p);   // the value pass runs with two 16-bit lanes

// K1m: a chain of value-only steps in which a big tensor absorbs small network
// tensors one after another, T_s = max(NEG, max over the labels step s sums of
// T_{s-1} + B_s), computed in one pass: C[y] = max over every label the chain sums
// of the left fold acc = max(acc + B_s, NEG) starting from A (max-plus addition
// distributes over max and both it and the floor are monotone, so this is the
// step-by-step result exactly, infeasible entries included). A is read once and C
// written once, where the separate steps read and write every intermediate.
constexpr int kChainMaxSteps = 8;     // B operands of one chain (4-bit index fields of a 32-bit word)
constexpr int kChainMaxSum = 3;       // labels summed inside one chain
struct ChainParams {
    const int32_t *a = nullptr;       // A value plane, fixed-variable offset applied
    int32_t *vc = nullptr;
    int rc = 0, rs = 0, L = 0;
    int8_t oA[32];                    // A bit of output bit i (-1: not in A)
    int8_t sA[kChainMaxSum];          // A bit of summed label j (-1: not in A)
    uint32_t wC[32];                  // output bit i's contribution to the packed B index word
    uint32_t wS[kChainMaxSum];        // summed label j's contribution (field s: bits 4s..4s+3 index B_s)
    const int32_t *b[kChainMaxSteps]; // B_s values, fixed-variable offset applied (<= 16 entries)
    int8_t bsize_log2[kChainMaxSteps];
};
// All entries must have the same L (1 <= L <= kChainMaxSteps) and rc >= 2.
cudaError_t launch_chain_batch(const ChainParams *p, int n, cudaStream_t s);

// out bit q <- in bit perm[q] (K2: shared-memory gather kernel)
cudaError_t launch_permute(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin,
                           uint64_t plane_in, int32_t *vout, uint64_t *cout, uint64_t plane_out,
                           int np, cudaStream_t s);
// K2t: the same with TMA tile loads and stores, for permutations whose output bits
// form at most five runs of consecutive input bits (the runs at input bit 0 and at
// output bit 0 of length 2 or more) on 16-byte aligned buffers.
bool permute_tma_eligible(int r, const int32_t *perm, const void *vin, const void *cin, uint64_t plane_in,
                          const void *vout, const void *cout, uint64_t plane_out, int np);
cudaError_t launch_permute_tma(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin, uint64_t plane_in,
                               int32_t *vout, uint64_t *cout, uint64_t plane_out, int np, cudaStream_t s);
// Whether a K2t block gave up waiting for a tile (and clears the flag). Synchronous.
cudaError_t permute_tma_timed_out(bool *flag);

// counting-(+) over n scalars (count plane t of the inputs at cnts + t*plane);
// result count t at out_cnt[t * out_plane]; scratch: aggregate_scratch_bytes(n, np)
size_t aggregate_scratch_bytes(int64_t n, int np);
cudaError_t launch_aggregate(int64_t n, const int32_t *vals, const uint64_t *cnts, uint64_t plane,
                             int np, const uint32_t *cprime, int32_t *out_val, uint64_t *out_cnt,
                             uint64_t out_plane, void *scratch, cudaStream_t s);

// K5: small subtrees of a contraction tree run by one thread block each, with every
// intermediate in shared memory and only the subtree's result written to global
// memory. One launch runs all subtrees of a plan.
constexpr int kFusedMaxBits = 16;      // output / summed bits of a fused step
struct FStep {
    int8_t rc, rs, hasB;
    int8_t a_kind, b_kind;             // 0: network tensor (global, unit counts), 1: shared memory
    int8_t c_kind;                     // 1: shared memory, 2: arena block, 3: external result
    int8_t a_rank, b_rank;             // ranks of shared-memory operands (plane stride 2^rank)
    int8_t oA[kFusedMaxBits], oB[kFusedMaxBits], sA[kFusedMaxBits], sB[kFusedMaxBits];
    uint32_t a_off, b_off, c_off;      // network: element offset (base included); smem: byte offset
    uint64_t c_goff;                   // arena byte offset (c_kind 2)
};
struct FSub {
    int first, count;                  // its steps, in post-order
    int leaf;                          // leaf sub-network: arena + leaf * arena_stride, out_* + leaf
};
struct FusedParams {
    const FStep *steps;
    const FSub *subs;
    int nsubs;
    const int32_t *net;
    char *arena;
    uint64_t arena_stride;             // bytes between the arenas of consecutive leaves
    int32_t *out_val;
    uint64_t *out_cnt;
    uint64_t out_plane;
    int np;
    uint32_t cprime[kMaxPlanes];
};
// byte offset of the count planes inside a shared-memory tensor of rank r
__host__ __device__ inline uint32_t smem_count_offset(int r) { return ((4u << r) + 15u) & ~15u; }
__host__ __device__ inline uint32_t smem_tensor_bytes(int r, int np) {
    return smem_count_offset(r) + (uint32_t)np * (8u << r);
}
cudaError_t launch_fused(const FusedParams &p, size_t smem_bytes, cudaStream_t s);

// Tropical argmax of one step for q selected outputs (values only).
struct BackwardParams {
    const int32_t *va = nullptr, *vb = nullptr, *vc = nullptr;
    uint64_t baseA = 0, baseB = 0;
    int rc = 0, rs = 0, hasB = 0;
    int8_t oA[32], oB[32], sA[32], sB[32];
};
cudaError_t launch_backward(const BackwardParams &p, int64_t q, const int64_t *sel_o,
                            int64_t *sel_a, int64_t *sel_b, cudaStream_t s);

// Fill a value plane with v and np count planes with c (initialisation helper).
cudaError_t launch_fill(int32_t *val, uint64_t *cnt, uint64_t n, uint64_t plane, int np,
                        int32_t v, uint64_t c, cudaStream_t s);

}  // namespace bbtn

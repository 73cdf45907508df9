/*
 * bbtn.h -- C ABI of the GB300 (sm_103a) Branch-and-Bound Tensor Network library.
 *
 * Method: Wang, Gao, Zhang, Pan, Liu, "Branch-and-Bound Tensor Networks for Exact
 * Ground-State Characterization", arXiv:2602.05470.
 *
 * The library contracts tropical tensor networks over the counting max-plus
 * semiring. Every tensor element is an int32 value plus an exact degeneracy count
 * carried in up to BBTN_MAX_PRIMES count planes of uint64 words: one residue per
 * word modulo a prime 2^61 - c (bbtn_primes), or two residues per word modulo a
 * pair of primes 2^30 - d (bbtn_prime_pairs; the solver's default).
 *
 * Conventions shared by every call
 *  - Return value: BBTN_OK (0) or a negative BBTN_E* code; bbtn_last_error() gives
 *    a message for the calling thread's most recent failure.
 *  - Semiring (paper Eq. (2) and the counting paragraph after it, in max-plus
 *    form): (a, c) (+) (b, d) = (max(a,b), c + d if a == b else the count of the
 *    larger); (a, c) (x) (b, d) = (a + b, c * d). The paper's min-sum network for an
 *    energy H is contracted as the max-plus network of -H. "-infinity" (the hard
 *    constraint (inf, 0) of the MWIS paragraph) is the value BBTN_NEG with count 0;
 *    every contraction floors values at BBTN_NEG, and any value below
 *    BBTN_FINITE_MIN is infeasible.
 *  - Tensors are over binary variables. A tensor of rank r has 2^r elements; bit i
 *    of the linear index is the value of variable labels[i] (labels are caller-
 *    chosen non-negative ints). Storage is structure-of-arrays: an int32 value
 *    plane of 2^r entries and np uint64 count planes, plane t at count + t*2^r.
 *  - "Device pointer" arguments must point to memory of the current CUDA device;
 *    "host" arguments to host memory. The caller owns every buffer it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device-level calls are asynchronous on that stream unless stated otherwise.
 */
#ifndef BBTN_H
#define BBTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BBTN_OK 0
#define BBTN_EINVAL (-1)     /* bad argument */
#define BBTN_ENOMEM (-2)     /* out of memory, or the space cap cannot be met */
#define BBTN_EOVERFLOW (-3)  /* degeneracy may exceed the CRT range: use more primes */
#define BBTN_ETIMEOUT (-4)   /* a bounded device wait gave up */
#define BBTN_EIO (-5)        /* file could not be read or parsed */
#define BBTN_ECUDA (-6)      /* a CUDA runtime call failed */
#define BBTN_ESTATE (-7)     /* call out of order (e.g. result before solve) */

#define BBTN_NEG (-(1 << 29))           /* -infinity sentinel (value plane) */
#define BBTN_FINITE_MIN (-(1 << 28))    /* values below this are infeasible */
#define BBTN_MAX_PRIMES 8
#define BBTN_MAX_RANK 30

/* ------------------------------------------------------------------ library info */

/* Version string of the library build. */
const char *bbtn_version(void);

/* Message of the calling thread's last failure ("" if none). Never NULL. */
const char *bbtn_last_error(void);

/* Size in bytes of the structures this header declares, so that a binding can check
 * its own copies of them: which = 0 bbtn_opts, 1 bbtn_stats, 2 bbtn_plan_info.
 * Returns 0 for any other value. */
size_t bbtn_struct_size(int which);

/* The first n primes used for count residues, written to primes[0..n-1] (host).
 * p_t = 2^61 - c_t, c_t ascending, each proven prime by deterministic
 * Miller-Rabin at library load. n <= BBTN_MAX_PRIMES + 1 (the last one is the
 * check prime used by the overflow guard). */
int bbtn_primes(int n, uint64_t *primes);

/* The first n pair moduli, written to moduli[0..n-1] (host): moduli[t] =
 * q[2t+1] << 32 | q[2t] for the primes q = 2^30 - d, d ascending. A count plane
 * with a pair modulus holds two residues per uint64 word: the low 32 bits mod
 * q[2t], the high 32 bits mod q[2t+1] (each half below its prime). The solver's
 * count planes take this form unless opts.wide_counts is set: a product of two
 * words is then two 32 x 32-bit multiplies instead of one 64 x 64 -> 128-bit one.
 * n <= BBTN_MAX_PRIMES + 1 (the last one is the check plane's). */
int bbtn_prime_pairs(int n, uint64_t *moduli);

/*
 * Chinese-remainder recombination (Garner's method) of k residues res[t] mod
 * distinct primes primes[t] (host arrays) into the unique integer in
 * [0, prod primes) as a decimal string -- the step that turns the per-prime
 * counts of the paper's counting algebra into the exact degeneracy. Host only.
 * *needed receives strlen + 1; buf may be NULL to query. Residues must be below
 * their primes.
 */
int bbtn_crt_decimal(int k, const uint64_t *res, const uint64_t *primes, char *buf, size_t cap,
                     size_t *needed);

/*
 * Integer-ALU throughput microbenchmark (measurement only; the paper has no
 * counterpart): the denominator of the register-tiled kernel's roofline. Runs
 * blocks x threads threads (threads a multiple of 32, at most 256), each with 8
 * independent dependency chains of `iters` x 4 add+max instructions: which = 0
 * __viaddmax_s32 (one tropical multiply-add each), 1 __viaddmax_s16x2 (two).
 * *ops receives the tropical multiply-adds executed and *ms the kernel's time
 * (CUDA events on `stream`). Blocking; allocates and frees a small device buffer.
 */
int bbtn_bench_alu(int which, int blocks, int threads, int iters, double *ops, float *ms, void *stream);

/* -------------------------------------------------------- device-level operations */
/*
 * One counting-tropical pairwise contraction (paper Eq. (2), one binary step of
 * contract(T)), computed entirely on the device:
 *     C[lc] = max(BBTN_NEG, max_s A[la] + B[lb]),  s = (la U lb) \ lc,
 *     cC_t[lc] = sum over maximising s of cA_t * cB_t  (mod p_t),  t < np.
 * la, lb, lc: host int arrays of ra, rb, rc distinct labels; every label of lc
 * must occur in la or lb. Labels in la or lb but not in lc are summed (labels
 * private to one operand included). rb = 0 with lb/vb/cb NULL makes B the
 * scalar (0, 1): a single-operand reduction.
 * va, vb, vc: device int32 value planes; ca, cb, cc: device uint64 count planes
 * (np planes each; unused when np == 0, the value-only mode). primes: host array of
 * np plane moduli, either all primes of the form 2^61 - c with c < 2^10 (as returned
 * by bbtn_primes; one residue per word) or all pair moduli (as returned by
 * bbtn_prime_pairs; two residues per word). Input counts must already be reduced
 * (each residue below its prime). Output buffers must not alias
 * inputs. Ranks up to BBTN_MAX_RANK. Asynchronous on `stream`.
 */
int bbtn_contract(int ra, const int32_t *la, const int32_t *va, const uint64_t *ca,
                  int rb, const int32_t *lb, const int32_t *vb, const uint64_t *cb,
                  int rc, const int32_t *lc, int32_t *vc, uint64_t *cc,
                  int np, const uint64_t *primes, void *stream);

/*
 * Bit permutation of a rank-r tensor (the layout change in front of a pairwise
 * step): out[j] = in[i] where bit perm[q] of i equals bit q of j, i.e. output bit
 * q is input bit perm[q]. perm: host array, a permutation of 0..r-1. Copies the
 * value plane and np count planes (device pointers, no aliasing).
 */
int bbtn_permute(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin,
                 int32_t *vout, uint64_t *cout, int np, void *stream);

/*
 * 1 if bbtn_permute with these arguments takes the TMA-staged kernel, else 0 (host
 * only; the pointers are only checked for alignment). That kernel moves tiles with
 * cp.async.bulk.tensor loads and stores through shared memory; it serves
 * permutations whose output bits form at most five runs of consecutive input bits
 * (the run at input bit 0 and the run at output bit 0 at least two bits long), on
 * 16-byte aligned buffers. bbtn_permute then synchronises `stream` before it
 * returns, to report a tile wait that gave up as BBTN_ETIMEOUT; other permutations
 * run the shared-memory gather kernel asynchronously.
 */
int bbtn_permute_uses_tma(int r, const int32_t *perm, const void *vin, const void *cin, const void *vout,
                          const void *cout, int np);

/*
 * Counting-(+) over n scalars (branch aggregation, paper: the final result is
 * the sum of the contractions of each branch): v* = max_b v_b and
 * c*_t = sum over b with v_b == v* of c_{b,t} mod p_t. vals: device int32[n];
 * counts: device uint64[np][n] (plane t at counts + t*n); out_val: device int32[1];
 * out_counts: device uint64[np]. n == 0 gives (BBTN_NEG, 0). Uses scratch memory
 * from the library's stream-ordered pool. Asynchronous on `stream`.
 */
int bbtn_aggregate(int64_t n, const int32_t *vals, const uint64_t *counts, int np,
                   const uint64_t *primes, int32_t *out_val, uint64_t *out_counts,
                   void *stream);

/*
 * The same reduction as bbtn_aggregate (same arguments, same result) but it
 * allocates nothing: no cudaMalloc, cudaFree or other allocating routine is called.
 * (The paper has no counterpart; this entry point exists for callers that must not
 * allocate while they run, e.g. an application whose own memory manager already
 * holds the whole device, or a latency-critical loop that keeps allocation out of
 * its steady state.) Its per-block partial results live in one fixed device array
 * of bbtn_aggregate_noalloc_max_scratch() bytes (64 KiB) compiled into the library;
 * every GPU that loads the library holds that array until the process exits. The
 * reduction never needs more than that for any n (at most 608 partials of up to
 * 9 planes), and a request that would is rejected with BBTN_EINVAL. The first call
 * on a device looks up the array's device address with that device current, so
 * make that first call before any stream capture. The address is looked up once per
 * device for the life of the process: after cudaDeviceReset on that device it is
 * stale, so do not call this entry point again on that device in the same process
 * (bbtn_aggregate has no such limit). All calls on a device share the
 * array and the last call's partials stay in it; nothing in it has to start at
 * zero, but calls that overlap on the GPU (concurrent streams) race on it.
 */
int bbtn_aggregate_noalloc(int64_t n, const int32_t *vals, const uint64_t *counts, int np,
                           const uint64_t *primes, int32_t *out_val, uint64_t *out_counts,
                           void *stream);
size_t bbtn_aggregate_noalloc_max_scratch(void);

/*
 * A chain of value-only pairwise steps in one pass (paper Eq. (2) applied L times,
 * no counts): T_0 = A, T_l = max(BBTN_NEG, max over the labels of T_{l-1} and B_l
 * missing from lc_l of T_{l-1} + B_l) with labels lc_l, and the result vc = T_L.
 * Every entry equals what L calls of bbtn_contract (np = 0) give, infeasible
 * entries included; A is read once and vc written once, and no intermediate is
 * stored. This is the step pattern in which a big frontier tensor absorbs edge
 * matrices one after another.
 * la: host int[ra] labels of A (va: device int32[2^ra]). L: 1..8 steps. rb: host
 * int[L], ranks 0..4 of the B_l; lb: host labels of B_0..B_{L-1} concatenated; vb:
 * host array of L device pointers (int32[2^rb[l]] each, never NULL). rc: host
 * int[L] ranks of the step results; lc: host labels of the results concatenated;
 * every label of lc_l must be in T_{l-1} or B_l. vc: device int32[2^rc[L-1]], not
 * aliasing an input. The chain must fit the fused kernel -- at most 3 labels summed
 * over the whole chain, 2^summed * L <= 16, final rank 2..30 -- else BBTN_EINVAL
 * (run the steps with bbtn_contract instead). Asynchronous on `stream`.
 */
int bbtn_contract_chain(int ra, const int32_t *la, const int32_t *va, int L, const int32_t *rb,
                        const int32_t *lb, const int32_t *const *vb, const int32_t *rc, const int32_t *lc,
                        int32_t *vc, void *stream);

/*
 * Value-only variant of bbtn_contract (same step, paper Eq. (2), no counts) for
 * operands whose finite values all lie in (-2^12, 2^12): the register-tiled
 * kernel then adds and maxes two 16-bit lanes per instruction (the solver uses
 * this for its value-only leaves when the instance's total value range allows
 * it). Every feasible output (>= BBTN_FINITE_MIN) equals bbtn_contract's; an
 * infeasible output is some value below BBTN_FINITE_MIN (BBTN_NEG from the 16-bit
 * kernel). Finite inputs outside the range give undefined feasible results.
 * Arguments as for bbtn_contract with np = 0; device pointers; asynchronous.
 */
int bbtn_contract_values16(int ra, const int32_t *la, const int32_t *va, int rb, const int32_t *lb,
                           const int32_t *vb, int rc, const int32_t *lc, int32_t *vc, void *stream);

/*
 * Tropical back-propagation through one pairwise step (the backward pass that
 * recovers an optimal configuration): for each of `q` selected output entries
 * sel_o[i] of C = contract(A, B) (values only), find the smallest summed
 * assignment s (as an integer whose bit j is the j-th summed label, in the order
 * (la \ lc) then (lb \ (la U lc))) with A + B == C[sel_o[i]], and write the
 * matching linear indices of A and B to sel_a[i], sel_b[i]. sel_* are device
 * int64 arrays; entries whose C value is infeasible get -1. Values only: the
 * count planes are not read.
 */
int bbtn_contract_backward(int ra, const int32_t *la, const int32_t *va,
                           int rb, const int32_t *lb, const int32_t *vb,
                           int rc, const int32_t *lc, const int32_t *vc,
                           int64_t q, const int64_t *sel_o, int64_t *sel_a, int64_t *sel_b,
                           void *stream);

/* ------------------------------------------------------------ solver (host-driven) */

typedef struct bbtn_ctx bbtn_ctx;   /* opaque; owned by the library */

#define BBTN_MODE_PLAIN 0    /* one contraction of the whole network (no slicing) */
#define BBTN_MODE_SLICED 1   /* dynamic slicing until the space cap holds */
#define BBTN_MODE_BBTN 2     /* branch-and-bound tensor network */

typedef struct {
    int space_cap_log2;      /* T_target of Eq. (4), in elements per tensor (default 24) */
    int n_primes;            /* count planes, 0 (values only) .. BBTN_MAX_PRIMES (3): 60 bits of
                                degeneracy range each (61 with wide_counts) */
    uint64_t seed;           /* order finder / tie-breaking seed */
    int mode;                /* BBTN_MODE_* (default BBTN_MODE_BBTN) */
    int sa_iters;            /* simulated-annealing sweeps of the order finder (default 20) */
    int region_size;         /* branching-region size |R| (default 8) */
    int batch;               /* leaves contracted per batch (default 64) */
    int use_gnn;             /* use the learned scorers attached by bbtn_set_gnn (default 0) */
    int count_check;         /* overflow guard: -1 auto, 0 off, 1 on (default -1) */
    int use_symmetry;        /* spin-flip symmetry when every field is 0 (default 1) */
    int verbose;             /* progress to stderr (default 0) */
    int profile;             /* time every contraction launch with CUDA events (default 0);
                                with the environment variable BBTN_PROFILE_DUMP set to a
                                path, a profiled solve also writes one CSV row per launch
                                there (operand and output ranks, summed labels, algorithmic
                                bytes and ops, milliseconds, kernel kind, leaves batched) */
    int max_slices_log2;     /* sliced mode: refuse more than 2^this slices (default 30) */
    int branch_lookahead;    /* seed of each branching region: the variable, among the this-many
                                carrying the most overflow, whose branching has the smallest
                                gamma (default 1: the one carrying the most overflow) */
    int leaf_trials;         /* BBTN counting leaves: order-finder trials (host threads) for each
                                leaf's own contraction order, used when it fits the cap with less
                                work than the root order restricted to the leaf (default 0: always
                                the root order, which the min-fill root orders made as good on the
                                30x30 King's-subgraph workload, at no host time) */
    int autotune;            /* time the register-tiled kernel's four load layouts on the first
                                step of each shape class and keep the fastest for the context's
                                later solves (default 0: the bit-0 rule, which the tuned choice
                                matched on the 30x30 King's-subgraph workload) */
    int wide_counts;         /* 1: one residue mod a prime 2^61 - c per count word; 0 (default): two
                                residues mod primes 2^30 - d per word (bbtn_prime_pairs) */
    int slice_sample;        /* sliced mode, timing only: > 0 contracts just the first this-many of
                                the 2^|V_f| slices (paper, slicing cost estimates: the time of a few
                                slices times the number of slices); the value and count are then those
                                of the sampled slices, not of the instance; stats.slices_run counts
                                them (default 0: every slice) */
    int arena_budget_mb;     /* device memory the leaf arenas of one launch group may take, in MiB
                                (default 0: half of the device memory free when the solve starts,
                                divided among the solves running on the device at that moment); a
                                single leaf always gets the arena its plan needs */
    int no_chain_fusion;     /* 1: run every value-only step as its own launch instead of fusing
                                chains of steps in which a big tensor absorbs small network tensors
                                into one pass (default 0: fused; the results are identical) */
    int order_restarts;      /* root contraction order: this many annealed restarts (host
                                threads), every odd one started from a min-fill elimination order
                                with its own tie-breaking seed, 0..64 (default 0: four restarts,
                                one of them from min-fill). The results are identical; only the
                                tree, and so the work and the branching, change */
} bbtn_opts;

typedef struct {
    double t_total_s;        /* wall time of the last bbtn_solve */
    double t_plan_s;         /* host planning (orders, branching) */
    double t_device_s;       /* wall time spent waiting on device work */
    double tropical_ops;     /* sum over steps of 2^{|union of labels|} multiply-adds */
    double bytes_moved;      /* algorithmic bytes of all contraction steps */
    double kernel_ms;        /* device time of contraction kernels (CUDA events) */
    int64_t nodes;           /* branch-and-bound nodes expanded */
    int64_t leaves;          /* sub-networks contracted */
    int64_t pruned;          /* branches discarded by bounds */
    int64_t launches;        /* kernel launches */
    int64_t steps;           /* pairwise contraction steps executed */
    int sc_log2;             /* largest tensor contracted (log2 elements) */
    double tc_log2;          /* log2 of the time complexity of the plain network */
    double sc_plain_log2;    /* space complexity of the plain network (log2) */
    int slices_log2;         /* |V_f| of the sliced mode */
    /* per-launch CUDA-event timing of the contraction kernels (profile mode only) */
    double prof_ms;          /* summed device time of all contraction launches */
    double prof_bytes;       /* their algorithmic bytes */
    double prof_ops;         /* their multiply-adds */
    int64_t prof_launches;
    double prof_scount_ms;   /* streaming gather kernel, counting steps: device time, bytes, launches */
    double prof_scount_bytes;
    int64_t prof_scount_launches;
    double prof_stream_ms;   /* streaming gather kernel (K1/K3), value-only steps: device time,
                                bytes, launches */
    double prof_stream_bytes;
    int64_t prof_stream_launches;
    double prof_tiled_ms;    /* register-tiled kernel (K1t), value-only steps: device time,
                                multiply-adds, launches */
    double prof_tiled_ops;
    int64_t prof_tiled_launches;
    int64_t prof_tiled16_launches; /* of those, launches with two 16-bit lanes per instruction */
    double prof_tcount_ms;   /* register-tiled kernel (K1t), counting steps: device time,
                                multiply-adds, launches */
    double prof_tcount_ops;
    int64_t prof_tcount_launches;
    int64_t slices_run;      /* sliced mode: slices contracted (2^slices_log2 unless opts.slice_sample) */
    double prof_chain_ms;    /* fused chains of value-only streaming steps (K1m): device time, */
    double prof_chain_bytes; /* algorithmic bytes (A read once, the result written once), launches */
    int64_t prof_chain_launches;
    int64_t chains;          /* K1m chains launched (one per chain and leaf) */
    int64_t chained_steps;   /* pairwise steps those chains replaced */
    /* configuration recovery (want_config): intermediates the forward kept as checkpoints,
       intermediates the top-down walk recomputed, the most tensor bytes alive at once, what
       keeping every intermediate would take, and the byte budget it ran under */
    int64_t bwd_kept;
    int64_t bwd_recomputed;
    double bwd_peak_bytes;
    double bwd_keep_all_bytes;
    double bwd_budget_bytes;
    /* algorithmic bytes of the register-tiled launches (profile mode), value-only and
       counting steps: with prof_tiled_ops / prof_tcount_ops they give each kernel's
       arithmetic intensity, which decides whether HBM or the integer pipe bounds it */
    double prof_tiled_bytes;
    double prof_tcount_bytes;
} bbtn_stats;

/* Fill *opts with defaults. */
void bbtn_default_opts(bbtn_opts *opts);

/* Create a solver context on the current CUDA device. opts may be NULL (defaults). */
int bbtn_create(const bbtn_opts *opts, bbtn_ctx **out);
void bbtn_destroy(bbtn_ctx *ctx);

/* Use `stream` for all device work of this context (default: a private stream). */
int bbtn_set_stream(bbtn_ctx *ctx, void *stream);

/*
 * Give the context a caller-owned device workspace (for example a block allocated
 * by PyTorch's caching allocator). Intermediates are placed in it by the static
 * memory planner; a plan that needs more returns BBTN_ENOMEM. Without a workspace
 * the context allocates (and keeps) its own. ptr must stay valid until the context
 * is destroyed or another workspace is set.
 */
int bbtn_set_workspace(bbtn_ctx *ctx, void *ptr, size_t bytes);

/*
 * Load a +-J / Ising instance (paper Eq. (1)): H = sum_E -J_ij s_i s_j - sum_V h_i s_i.
 * n vertices 0..n-1, m edges; edges: host int32[2m] pairs; J: host int32[m];
 * h2: host int32[n] holding 2*h_i (NULL = no field). |J|, |h2| <= 2^16.
 */
int bbtn_load_spin_glass(bbtn_ctx *ctx, int n, int m, const int32_t *edges,
                         const int32_t *J, const int32_t *h2);

/*
 * Load a maximum-weight independent set instance (paper, MWIS paragraph):
 * weights w: host int32[n] in 1..2^16 (NULL = unit weights, plain MIS).
 */
int bbtn_load_mwis(bbtn_ctx *ctx, int n, int m, const int32_t *edges, const int32_t *w);

/* Load an instance file (plain text: "p spin|mwis n m", "e i j [J]", "f i h2", "w i w"). */
int bbtn_load_file(bbtn_ctx *ctx, const char *path);

/*
 * Solve the loaded instance. want_count: compute the exact degeneracy;
 * want_config: also recover one optimal configuration (tropical backward).
 * Blocking. Results stay valid until the next load or solve.
 */
int bbtn_solve(bbtn_ctx *ctx, int want_count, int want_config);

/*
 * Branch sharding across ranks (one process per GPU). The paper's final result is
 * the counting sum of the contractions of each branch (BBTN section), and the
 * leaves are independent sub-networks, so `world` ranks can split one instance's
 * leaves. Every rank loads the same instance into a context with the same options
 * (BBTN mode) and runs:
 *  1. bbtn_shard_values(ctx, rank, world, want_count, &local_max): expands the
 *     search tree on the host (only the heuristic incumbent prunes, so every rank
 *     gets the same leaf list) and contracts, values only, the leaves i with
 *     i mod world == rank. *local_max: the largest leaf maximum of this rank, in the
 *     library's max-plus convention (-2H for spin glasses, alpha for MWIS), or
 *     BBTN_NEG if none of its leaves is feasible.
 *  2. the caller takes global_max = the maximum of local_max over the ranks (one
 *     all-reduce);
 *  3. bbtn_shard_counts(ctx, global_max, want_config, ...): contracts with counts
 *     this rank's leaves whose maximum equals global_max and returns this rank's
 *     part of the counting sum: *value = global_max if it holds such a leaf, else
 *     BBTN_NEG; planes[t] (host uint64[*np]) its count in plane t, modulo moduli[t]
 *     (a pair word q1 << 32 | q0 or a 61-bit prime, as for bbtn_contract; the
 *     spin-flip factor already applied), zero with BBTN_NEG; *n_crt_planes planes
 *     enter the CRT, a further one (if *np is larger) is the overflow check. With
 *     want_config and an optimal leaf on this rank, config (host int8[n]) receives an
 *     optimal configuration (+-1 or 0/1) and *have_config = 1, else 0. Arrays of
 *     BBTN_MAX_PRIMES + 1 entries always suffice.
 *  4. the caller combines the ranks' (value, planes) by the counting sum
 *     (bbtn_aggregate over the gathered results, all with the same moduli) and turns
 *     the combined planes into the decimal count with bbtn_count_decimal.
 * With world == 1 this gives bbtn_solve's energy and count (a search whose leaves
 * are fixed in advance may contract more leaves than bbtn_solve, never fewer
 * optimal ones). The context holds the rank's leaf list between steps 1 and 3;
 * loading an instance or calling bbtn_solve on it in between discards it (step 3 then
 * returns BBTN_ESTATE).
 */
int bbtn_shard_values(bbtn_ctx *ctx, int rank, int world, int want_count, int64_t *local_max);
int bbtn_shard_counts(bbtn_ctx *ctx, int64_t global_max, int want_config, int32_t *value, uint64_t *planes,
                      uint64_t *moduli, int *np, int *n_crt_planes, int8_t *config, int *have_config);

/*
 * The exact degeneracy from np count-plane words (host): residues modulo the
 * planes' moduli (pair words split into their two residues), Garner CRT of the
 * first n_crt_planes planes into a decimal string (buf, cap; *needed = strlen + 1,
 * buf may be NULL to query). A further plane is the overflow check: if its
 * residues disagree with the CRT result, BBTN_EOVERFLOW. Host only.
 */
int bbtn_count_decimal(int np, int n_crt_planes, const uint64_t *planes, const uint64_t *moduli, char *buf,
                       size_t cap, size_t *needed);

/* 2*H* for a spin glass (so that half-integer fields stay integral); alpha for MWIS. */
int bbtn_get_energy(bbtn_ctx *ctx, int64_t *e);

/* Count residues: res[t] = D mod primes[t], t < *k, one per CRT prime (two per count
 * plane with pair moduli; host arrays of >= 2 * BBTN_MAX_PRIMES). */
int bbtn_get_count_residues(bbtn_ctx *ctx, uint64_t *res, uint64_t *primes, int *k);

/* Degeneracy D as a decimal string (CRT / Garner recombination of the residues).
 * *needed receives strlen + 1; buf may be NULL to query. */
int bbtn_get_count_dec(bbtn_ctx *ctx, char *buf, size_t cap, size_t *needed);

/* One optimal configuration: s[i] in {-1,+1} (spin glass) or {0,1} (MWIS). Host int8[n]. */
int bbtn_get_config(bbtn_ctx *ctx, int8_t *s);

/* Statistics of the last solve. */
int bbtn_get_stats(bbtn_ctx *ctx, bbtn_stats *st);

/* Host-side planning summary (no device work; usable without a GPU). */
typedef struct {
    double tc_log2;          /* log2 time complexity of the (unsliced) network's tree */
    int sc_log2;             /* its space complexity (largest tensor, log2 elements) */
    double rho;              /* Eq. (4) overflow of that tree at the space cap */
    int slices_log2;         /* |V_f| chosen by dynamic slicing (sliced mode, else 0) */
    int64_t steps;           /* pairwise steps of one leaf / slice */
    double ops;              /* its multiply-adds */
    double bytes;            /* its algorithmic bytes */
    double arena_bytes;      /* device arena the static memory plan needs */
    int64_t bb_nodes;        /* BBTN mode: nodes of the search tree, expanded on the host */
    int64_t bb_leaves;       /* BBTN mode: its leaf sub-networks */
    int chains;              /* fused chains of value-only steps in the step list (values-only plans) */
    int chained_steps;       /* the steps they replace */
    int bwd_kept;            /* configuration recovery of the root network under the budget
                                (opts.arena_budget_mb, else 1 GiB): checkpoints the forward keeps, */
    int bwd_recomputed;      /* intermediates the walk recomputes, */
    double bwd_peak_bytes;   /* tensor bytes alive at most, */
    double bwd_keep_all_bytes; /* and what keeping every intermediate takes */
} bbtn_plan_info;

/*
 * Plan the loaded instance on the host only: contraction order (and the slicing
 * set in sliced mode), and the step list of the first slice (all sliced variables
 * 0). In BBTN mode the whole search tree is also expanded on the host (no leaf is
 * contracted, so only the heuristic incumbent prunes) and its size reported; with
 * opts.use_gnn and a branch scorer attached, the scorer's forward passes run on
 * the device. If dump_path is not NULL, one CSV line per step is written there:
 * rank_a, rank_b, rank_c, summed, low_identity_bits, bytes, ops, nb, nm, nn (output bits in both
 * operands / only A / only B), node, a_node, b_node (tree nodes of the result and the operands),
 * fused (1 when the step runs inside the fused small-subtree kernel), chain (L on the last step of
 * a fused chain of L steps, -1 on its earlier steps, 0 elsewhere).
 */
int bbtn_analyze(bbtn_ctx *ctx, bbtn_plan_info *info, const char *dump_path);


/* ------------------------------------------------------------ learned branching (GNN) */
/*
 * A message-passing graph network that scores the vertices of a branch-and-bound
 * sub-problem. The paper's discussion names learned policies as the replacement for
 * its myopic branching heuristics; this model is that idea made concrete and has
 * no counterpart in the paper's experiments. It predicts, per free vertex, the
 * logit of x_v = 1 in an optimal configuration. The solver uses it (opts.use_gnn
 * with a model attached by bbtn_set_gnn, MWIS instances only) for a first
 * incumbent and for the order in which children are visited; it never prunes, so
 * energies and counts do not depend on it.
 *
 * Architecture (fp32, all kernels hand-written): input features X0 (n x 8);
 * three layers Z_l = H_{l-1} W_l + (A H_{l-1}) U_l + b_l, H_l = relu(Z_l) with
 * hidden width 64 and A the adjacency matrix; head s = H_3 w + c.
 * Loss: mean over masked vertices of softplus(s) - y s. Optimiser: Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameter vector (bbtn_gnn_param_count floats): for l = 1..3 W_l (din x 64,
 * row-major), U_l (din x 64), b_l (64), din = 8 for l = 1 else 64; then w (64), c.
 * Feature row of vertex v: [free, fixed to 0, fixed to 1, w_v / 10,
 * free neighbours / 8, degree / 8, neighbours fixed to 1 / 8, overflow share],
 * the overflow share being the variable's part of the Eq. (4) overflow of the
 * sub-network relative to the largest (0 where not given).
 *
 * Two roles (bbtn_set_gnn): a branch scorer picks the seed of each branching
 * region among the overflow-carrying variables (trained to imitate the lookahead
 * of opts.branch_lookahead, rows from bbtn_branch_samples); a value model predicts
 * an optimal configuration (first incumbent, order of children; MWIS only).
 */
typedef struct bbtn_gnn bbtn_gnn;   /* opaque; owns its device buffers */

#define BBTN_GNN_FEATURES 8

/* Create a model on the current device with Glorot-uniform weights from `seed`. */
int bbtn_gnn_create(uint64_t seed, bbtn_gnn **out);
void bbtn_gnn_destroy(bbtn_gnn *g);
int bbtn_gnn_param_count(void);
/* Use `stream` for the model's device work (default: the legacy stream). */
int bbtn_gnn_set_stream(bbtn_gnn *g, void *stream);

/*
 * Host-side feature rows (n x BBTN_GNN_FEATURES floats, row-major, into out) of a
 * graph with n vertices and m edges (host int32[2m]); w: host int32[n] vertex
 * weights (NULL = 1); fixed: host int8[n], -1 free, 0 or 1 fixed (NULL = all free);
 * score: host float[n] overflow shares (NULL = 0).
 */
int bbtn_gnn_features(int n, int m, const int32_t *edges, const int32_t *w, const int8_t *fixed,
                      const float *score, float *out);

/* Set the graph the next forward / train calls run on (uploads CSR lists). */
int bbtn_gnn_set_graph(bbtn_gnn *g, int n, int m, const int32_t *edges);

/* Logits of every vertex: feats host float[n*8] -> scores host float[n]. Blocking. */
int bbtn_gnn_forward(bbtn_gnn *g, const float *feats, float *scores);

/*
 * Forward + backward of the masked loss, then one Adam step with learning rate
 * lr (lr <= 0: gradients only, parameters unchanged). labels, mask: host
 * float[n] (labels in {0,1}; mask 0 or 1, the mean runs over mask-1 vertices).
 * *loss receives the loss before the step. Blocking.
 */
int bbtn_gnn_train_step(bbtn_gnn *g, const float *feats, const float *labels, const float *mask, float lr,
                        float *loss);

/* Copy parameters / the last gradients (host float[bbtn_gnn_param_count()]).
 * set_params also resets the Adam moments. */
int bbtn_gnn_get_params(bbtn_gnn *g, float *p);
int bbtn_gnn_set_params(bbtn_gnn *g, const float *p);
int bbtn_gnn_get_grads(bbtn_gnn *g, float *grad);

/* Attach models to a solver context (borrowed; NULL detaches that role). Used
 * when opts.use_gnn is set. They must outlive their use by bbtn_solve. */
int bbtn_set_gnn(bbtn_ctx *ctx, bbtn_gnn *branch_scorer, bbtn_gnn *value_model);

/*
 * Training rows for the branch scorer: expands the search tree of the loaded
 * instance on the host (as bbtn_analyze in BBTN mode, seeds chosen by a lookahead
 * over `lookahead` candidates) and records up to max_rows expanded nodes: fx
 * (int8[max_rows*n], -1 free / 0 / 1), score (float[max_rows*n], overflow share)
 * and gamma (float[max_rows*n]: the branching factor of the region seeded at that
 * variable; -1 for variables that carry no overflow, 0 where the region admits no
 * feasible configuration). *rows receives the rows written. Host only.
 */
int bbtn_branch_samples(bbtn_ctx *ctx, int max_rows, int lookahead, int8_t *fx, float *score, float *gamma,
                        int *rows);

/*
 * Host-only preparation of the loaded instance: builds its network and finds the
 * root contraction order with ctx's options, leaving the order in a process-wide
 * cache (keyed by the network's tensor labels, the root's fixed variables and the
 * order-finder settings; at most 256 entries). A later bbtn_solve of an instance
 * with the same structure and options, in any context, reuses it. Thread-safe with
 * respect to solves on other contexts, so the order of the next instance can be
 * found while the current one runs on the device. Uses no GPU.
 */
int bbtn_prepare(bbtn_ctx *ctx);

/* Empties the process-wide cache of root contraction orders (e.g. to time solves
 * that find their orders themselves). */
int bbtn_clear_order_cache(void);

/*
 * The leaf sub-networks of the branch-and-bound search of the loaded instance,
 * expanded on the host as bbtn_analyze does (BBTN section: the leaves are the
 * branches whose contractions are summed; only the heuristic incumbent prunes).
 * Writes the fixings of the first min(max_leaves, leaves) leaves to fx (host
 * int8[max_leaves * n], row per leaf: -1 free, 0 or 1 fixed) and the number of
 * leaves of the whole search to *leaves. Host only.
 */
int bbtn_search_leaves(bbtn_ctx *ctx, int64_t max_leaves, int8_t *fx, int64_t *leaves);

#ifdef __cplusplus
}
#endif
#endif /* BBTN_H */

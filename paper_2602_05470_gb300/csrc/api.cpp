// extern "C" entry points declared in include/bbtn.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "../../include/bbtn.h"
#include "common.h"
#include "exec.h"
#include "gnn.h"
#include "kernels.h"
#include "network.h"
#include "solver.h"

using namespace bbtn;

struct bbtn_ctx {
    bbtn_opts opts;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    Problem prob;
    bool loaded = false;
    bool solved = false;
    SolveOutput out;
    bbtn_stats stats;
    Arena arena;
    TileTuner tuner;                   // tuned load layouts, kept across solves
    GnnModel *gnn_branch = nullptr;   // borrowed (bbtn_set_gnn)
    GnnModel *gnn_value = nullptr;
    std::unique_ptr<Solver> shard;     // branch sharding between bbtn_shard_values and bbtn_shard_counts
};

namespace {

template <class F>
int guarded(F &&f) {
    try {
        f();
        set_error("");
        return BBTN_OK;
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host out of memory");
        return BBTN_ENOMEM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return BBTN_EINVAL;
    }
}

void check_labels(int r, const int32_t *l, const char *what) {
    if (r < 0 || r > BBTN_MAX_RANK) fail(BBTN_EINVAL, std::string(what) + ": rank out of range");
    if (r > 0 && !l) fail(BBTN_EINVAL, std::string(what) + ": labels missing");
    for (int i = 0; i < r; i++) {
        if (l[i] < 0) fail(BBTN_EINVAL, std::string(what) + ": negative label");
        for (int j = 0; j < i; j++)
            if (l[i] == l[j]) fail(BBTN_EINVAL, std::string(what) + ": repeated label");
    }
}

int find(int r, const int32_t *l, int x) {
    for (int i = 0; i < r; i++) if (l[i] == x) return i;
    return -1;
}

void cprimes_from(int np, const uint64_t *primes, uint32_t *c) { plane_moduli(np, primes, c); }

}  // namespace

extern "C" {

const char *bbtn_version(void) { return "bbtn-gb300 0.1 (sm_103a)"; }

const char *bbtn_last_error(void) { return get_error(); }

size_t bbtn_struct_size(int which) {
    switch (which) {
        case 0: return sizeof(bbtn_opts);
        case 1: return sizeof(bbtn_stats);
        case 2: return sizeof(bbtn_plan_info);
        default: return 0;
    }
}

int bbtn_primes(int n, uint64_t *primes) {
    return guarded([&] {
        const auto &tab = prime_table();
        if (n < 0 || n > (int)tab.size() || (n > 0 && !primes)) fail(BBTN_EINVAL, "bad prime count");
        for (int i = 0; i < n; i++) primes[i] = tab[i];
    });
}

int bbtn_prime_pairs(int n, uint64_t *moduli) {
    return guarded([&] {
        const auto &tab = pair_prime_table();
        if (n < 0 || 2 * n > (int)tab.size() || (n > 0 && !moduli)) fail(BBTN_EINVAL, "bad pair count");
        for (int i = 0; i < n; i++) moduli[i] = tab[2 * i + 1] << 32 | tab[2 * i];
    });
}

int bbtn_crt_decimal(int k, const uint64_t *res, const uint64_t *primes, char *buf, size_t cap,
                     size_t *needed) {
    return guarded([&] {
        if (k < 1 || k > 64 || !res || !primes) fail(BBTN_EINVAL, "bad residue list");
        std::vector<uint64_t> r(res, res + k), p(primes, primes + k);
        for (int t = 0; t < k; t++) {
            if (!is_prime_u64(p[t])) fail(BBTN_EINVAL, "moduli must be primes");
            if (r[t] >= p[t]) fail(BBTN_EINVAL, "residue not below its modulus");
            for (int u = 0; u < t; u++) if (p[u] == p[t]) fail(BBTN_EINVAL, "repeated modulus");
        }
        std::string s = crt_decimal(r, p);
        if (needed) *needed = s.size() + 1;
        if (buf) {
            if (cap < s.size() + 1) fail(BBTN_EINVAL, "buffer too small");
            memcpy(buf, s.c_str(), s.size() + 1);
        }
    });
}

namespace {

int contract_impl(int ra, const int32_t *la, const int32_t *va, const uint64_t *ca, int rb, const int32_t *lb,
                  const int32_t *vb, const uint64_t *cb, int rc, const int32_t *lc, int32_t *vc, uint64_t *cc,
                  int np, const uint64_t *primes, int v16, void *stream) {
    return guarded([&] {
        check_labels(ra, la, "A");
        check_labels(rb, lb, "B");
        check_labels(rc, lc, "C");
        if (!va || !vc) fail(BBTN_EINVAL, "value planes missing");
        if (rb > 0 && !vb) fail(BBTN_EINVAL, "B values missing");
        if (np > 0 && !cc) fail(BBTN_EINVAL, "C counts missing");
        ContractParams P;
        cprimes_from(np, primes, P.cprime);
        for (int i = 0; i < 32; i++) P.oA[i] = P.oB[i] = P.sA[i] = P.sB[i] = -1;
        for (int i = 0; i < rc; i++) {
            int pa = find(ra, la, lc[i]), pb = find(rb, lb, lc[i]);
            if (pa < 0 && pb < 0) fail(BBTN_EINVAL, "output label not in A or B");
            P.oA[i] = (int8_t)pa;
            P.oB[i] = (int8_t)pb;
        }
        int rs = 0;
        for (int i = 0; i < ra; i++)
            if (find(rc, lc, la[i]) < 0) {
                if (rs >= 32) fail(BBTN_EINVAL, "more than 32 summed labels");
                P.sA[rs] = (int8_t)i;
                P.sB[rs] = (int8_t)find(rb, lb, la[i]);
                rs++;
            }
        for (int i = 0; i < rb; i++)
            if (find(rc, lc, lb[i]) < 0 && find(ra, la, lb[i]) < 0) {
                if (rs >= 32) fail(BBTN_EINVAL, "more than 32 summed labels");
                P.sA[rs] = -1;
                P.sB[rs] = (int8_t)i;
                rs++;
            }
        P.rc = rc;
        P.rs = rs;
        P.np = np;
        P.v16 = v16;
        P.hasB = rb > 0 || vb != nullptr;
        P.A.val = va;
        P.A.cnt = ca;
        P.A.plane = 1ull << ra;
        P.A.unit_counts = ca == nullptr;
        if (P.hasB) {
            P.B.val = vb;
            P.B.cnt = cb;
            P.B.plane = 1ull << rb;
            P.B.unit_counts = cb == nullptr;
        }
        P.vc = vc;
        P.cc = cc;
        P.planeC = 1ull << rc;
        cudaStream_t s = (cudaStream_t)stream;
        void *scratch = nullptr;
        size_t sb = 0;
        if (splitk_eligible(P)) {   // few outputs, long sums: split-K needs a small scratch
            sb = splitk_scratch_bytes(rc, np);
            BBTN_CUDA(cudaMallocAsync(&scratch, sb, s));
        }
        cudaError_t e = launch_contract(P, s, nullptr, scratch, sb);
        if (scratch) cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("contract: ") + cudaGetErrorString(e));
    });
}

}  // namespace

int bbtn_contract_chain(int ra, const int32_t *la, const int32_t *va, int L, const int32_t *rb, const int32_t *lb,
                        const int32_t *const *vb, const int32_t *rc, const int32_t *lc, int32_t *vc, void *stream) {
    return guarded([&] {
        check_labels(ra, la, "A");
        if (L < 1 || L > kChainMaxSteps || !rb || !rc || !vb || !va || !vc) fail(BBTN_EINVAL, "bad chain arguments");
        std::vector<int> labA(la, la + ra);
        std::vector<std::vector<int>> labB(L), labC(L);
        const int32_t *pb = lb, *pc = lc;
        std::vector<int> prev = labA;
        for (int l = 0; l < L; l++) {
            if (rb[l] < 0 || rb[l] > 4 || !vb[l] || (rb[l] > 0 && !pb))
                fail(BBTN_EINVAL, "chain: B rank outside 0..4 or B missing");
            check_labels(rb[l], pb, "B");
            check_labels(rc[l], pc, "C");
            labB[l].assign(pb, pb + rb[l]);
            labC[l].assign(pc, pc + rc[l]);
            for (int x : labC[l])
                if (std::find(prev.begin(), prev.end(), x) == prev.end() &&
                    std::find(labB[l].begin(), labB[l].end(), x) == labB[l].end())
                    fail(BBTN_EINVAL, "chain: an output label is in neither operand of its step");
            prev = labC[l];
            pb += rb[l];
            pc += rc[l];
        }
        ChainParams cp;
        if (!chain_params(labA, labB, labC, cp))
            fail(BBTN_EINVAL, "chain does not fit the fused kernel (at most 8 steps, 3 summed labels over the chain, "
                              "2^summed * steps <= 16, output rank 2..30)");
        cp.a = va;
        cp.vc = vc;
        for (int l = 0; l < L; l++) cp.b[l] = vb[l];
        cudaError_t e = launch_chain_batch(&cp, 1, (cudaStream_t)stream);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("chain: ") + cudaGetErrorString(e));
    });
}

int bbtn_contract(int ra, const int32_t *la, const int32_t *va, const uint64_t *ca, int rb,
                  const int32_t *lb, const int32_t *vb, const uint64_t *cb, int rc, const int32_t *lc,
                  int32_t *vc, uint64_t *cc, int np, const uint64_t *primes, void *stream) {
    return contract_impl(ra, la, va, ca, rb, lb, vb, cb, rc, lc, vc, cc, np, primes, 0, stream);
}

int bbtn_contract_values16(int ra, const int32_t *la, const int32_t *va, int rb, const int32_t *lb,
                           const int32_t *vb, int rc, const int32_t *lc, int32_t *vc, void *stream) {
    return contract_impl(ra, la, va, nullptr, rb, lb, vb, nullptr, rc, lc, vc, nullptr, 0, nullptr, 1, stream);
}

int bbtn_permute_uses_tma(int r, const int32_t *perm, const void *vin, const void *cin, const void *vout,
                          const void *cout, int np) {
    if (r < 0 || r > BBTN_MAX_RANK || np < 0 || np > kMaxPlanes || (r > 0 && !perm)) return 0;
    return permute_tma_eligible(r, perm, vin, cin, 1ull << r, vout, cout, 1ull << r, np) ? 1 : 0;
}

int bbtn_permute(int r, const int32_t *perm, const int32_t *vin, const uint64_t *cin, int32_t *vout,
                 uint64_t *cout, int np, void *stream) {
    return guarded([&] {
        if (r < 0 || r > BBTN_MAX_RANK || np < 0 || np > kMaxPlanes) fail(BBTN_EINVAL, "bad rank / np");
        if (!vin || !vout || (np > 0 && (!cin || !cout)) || (r > 0 && !perm)) fail(BBTN_EINVAL, "null buffer");
        bool seen[32] = {false};
        for (int q = 0; q < r; q++) {
            if (perm[q] < 0 || perm[q] >= r || seen[perm[q]]) fail(BBTN_EINVAL, "perm is not a permutation");
            seen[perm[q]] = true;
        }
        cudaStream_t s = (cudaStream_t)stream;
        if (permute_tma_eligible(r, perm, vin, cin, 1ull << r, vout, cout, 1ull << r, np)) {
            cudaError_t e = launch_permute_tma(r, perm, vin, cin, 1ull << r, vout, cout, 1ull << r, np, s);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("permute (TMA): ") + cudaGetErrorString(e));
            // the tile waits are bounded: read back whether one gave up
            BBTN_CUDA(cudaStreamSynchronize(s));
            bool timed_out = false;
            BBTN_CUDA(permute_tma_timed_out(&timed_out));
            if (timed_out) fail(BBTN_ETIMEOUT, "permute (TMA): a tile load did not complete");
            return;
        }
        cudaError_t e = launch_permute(r, perm, vin, cin, 1ull << r, vout, cout, 1ull << r, np, s);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("permute: ") + cudaGetErrorString(e));
    });
}

int bbtn_aggregate(int64_t n, const int32_t *vals, const uint64_t *counts, int np, const uint64_t *primes,
                   int32_t *out_val, uint64_t *out_counts, void *stream) {
    return guarded([&] {
        if (n < 0 || !out_val || (n > 0 && !vals) || (np > 0 && (!out_counts || (n > 0 && !counts))))
            fail(BBTN_EINVAL, "bad aggregate arguments");
        uint32_t c[kMaxPlanes];
        cprimes_from(np, primes, c);
        cudaStream_t s = (cudaStream_t)stream;
        size_t sb = aggregate_scratch_bytes(n, np);
        void *scratch = nullptr;
        if (sb) BBTN_CUDA(cudaMallocAsync(&scratch, sb, s));
        cudaError_t e = launch_aggregate(n, vals, counts, (uint64_t)n, np, c, out_val, out_counts, 1, scratch, s);
        if (scratch) cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("aggregate: ") + cudaGetErrorString(e));
    });
}

int bbtn_contract_backward(int ra, const int32_t *la, const int32_t *va, int rb, const int32_t *lb,
                           const int32_t *vb, int rc, const int32_t *lc, const int32_t *vc, int64_t q,
                           const int64_t *sel_o, int64_t *sel_a, int64_t *sel_b, void *stream) {
    return guarded([&] {
        check_labels(ra, la, "A");
        check_labels(rb, lb, "B");
        check_labels(rc, lc, "C");
        if (q < 0 || (q > 0 && (!sel_o || !sel_a || !sel_b)) || !va || !vc) fail(BBTN_EINVAL, "bad arguments");
        BackwardParams B;
        for (int i = 0; i < 32; i++) B.oA[i] = B.oB[i] = B.sA[i] = B.sB[i] = -1;
        for (int i = 0; i < rc; i++) {
            int pa = find(ra, la, lc[i]), pb = find(rb, lb, lc[i]);
            if (pa < 0 && pb < 0) fail(BBTN_EINVAL, "output label not in A or B");
            B.oA[i] = (int8_t)pa;
            B.oB[i] = (int8_t)pb;
        }
        int rs = 0;
        for (int i = 0; i < ra; i++)
            if (find(rc, lc, la[i]) < 0) {
                B.sA[rs] = (int8_t)i;
                B.sB[rs] = (int8_t)find(rb, lb, la[i]);
                rs++;
            }
        for (int i = 0; i < rb; i++)
            if (find(rc, lc, lb[i]) < 0 && find(ra, la, lb[i]) < 0) {
                B.sA[rs] = -1;
                B.sB[rs] = (int8_t)i;
                rs++;
            }
        if (rs > 32) fail(BBTN_EINVAL, "more than 32 summed labels");
        B.rc = rc;
        B.rs = rs;
        B.hasB = rb > 0 || vb != nullptr;
        B.va = va;
        B.vb = vb;
        B.vc = vc;
        cudaError_t e = launch_backward(B, q, sel_o, sel_a, sel_b, (cudaStream_t)stream);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("backward: ") + cudaGetErrorString(e));
    });
}

void bbtn_default_opts(bbtn_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->space_cap_log2 = 24;
    o->n_primes = 3;
    o->seed = 1;
    o->mode = BBTN_MODE_BBTN;
    o->sa_iters = 20;
    o->region_size = 8;
    o->batch = 64;
    o->use_gnn = 0;
    o->count_check = -1;
    o->use_symmetry = 1;
    o->verbose = 0;
    o->profile = 0;
    o->max_slices_log2 = 30;
    o->branch_lookahead = 1;
    o->leaf_trials = 0;
    o->autotune = 0;
    o->wide_counts = 0;
    o->slice_sample = 0;
    o->arena_budget_mb = 0;
    o->no_chain_fusion = 0;
    o->order_restarts = 0;
}

int bbtn_create(const bbtn_opts *opts, bbtn_ctx **out) {
    return guarded([&] {
        if (!out) fail(BBTN_EINVAL, "out is NULL");
        auto ctx = std::make_unique<bbtn_ctx>();
        if (opts) ctx->opts = *opts;
        else bbtn_default_opts(&ctx->opts);
        const bbtn_opts &o = ctx->opts;
        if (o.space_cap_log2 < 1 || o.space_cap_log2 > 30) fail(BBTN_EINVAL, "space_cap_log2 outside 1..30");
        if (o.n_primes < 0 || o.n_primes > BBTN_MAX_PRIMES) fail(BBTN_EINVAL, "n_primes outside 0..8");
        if (o.mode < 0 || o.mode > 2) fail(BBTN_EINVAL, "unknown mode");
        if (o.region_size < 1 || o.region_size > 16) fail(BBTN_EINVAL, "region_size outside 1..16");
        if (o.batch < 1) fail(BBTN_EINVAL, "batch < 1");
        if (o.sa_iters < 0) fail(BBTN_EINVAL, "sa_iters < 0");
        if (o.branch_lookahead < 0 || o.branch_lookahead > 1024) fail(BBTN_EINVAL, "branch_lookahead outside 0..1024");
        if (o.leaf_trials < 0 || o.leaf_trials > 256) fail(BBTN_EINVAL, "leaf_trials outside 0..256");
        if (o.order_restarts < 0 || o.order_restarts > 64) fail(BBTN_EINVAL, "order_restarts outside 0..64");
        // without a usable device the context still plans on the host (bbtn_analyze);
        // every call that needs the device then fails with BBTN_ECUDA
        if (cudaGetDevice(&ctx->device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) == cudaSuccess) {
            ctx->own_stream = true;
        } else {
            cudaGetLastError();
            ctx->device = -1;
            ctx->stream = nullptr;
        }
        memset(&ctx->stats, 0, sizeof(ctx->stats));
        *out = ctx.release();
    });
}

void bbtn_destroy(bbtn_ctx *ctx) {
    if (!ctx) return;
    ctx->shard.reset();
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    ctx->arena.stream = ctx->stream;
    ctx->arena.release();
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int bbtn_set_stream(bbtn_ctx *ctx, void *stream) {
    return guarded([&] {
        if (!ctx) fail(BBTN_EINVAL, "ctx is NULL");
        // the arena is freed and regrown in stream order: finish the old stream's use of it first
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
        ctx->stream = (cudaStream_t)stream;
        ctx->arena.stream = ctx->stream;
        ctx->own_stream = false;
    });
}

int bbtn_set_workspace(bbtn_ctx *ctx, void *ptr, size_t bytes) {
    return guarded([&] {
        if (!ctx || (!ptr && bytes)) fail(BBTN_EINVAL, "bad workspace");
        if (!ptr) ctx->arena.release();
        else ctx->arena.adopt(ptr, bytes);
    });
}

static int load_common(bbtn_ctx *ctx, Problem &&p) {
    return guarded([&] {
        validate(p);
        ctx->shard.reset();   // a new instance discards a branch-sharded solve in progress
        ctx->prob = std::move(p);
        ctx->loaded = true;
        ctx->solved = false;
    });
}

int bbtn_load_spin_glass(bbtn_ctx *ctx, int n, int m, const int32_t *edges, const int32_t *J,
                         const int32_t *h2) {
    if (!ctx || n < 1 || m < 0 || (m > 0 && (!edges || !J))) {
        set_error("bad arguments to bbtn_load_spin_glass");
        return BBTN_EINVAL;
    }
    Problem p;
    p.kind = kSpin;
    p.n = n;
    for (int k = 0; k < m; k++) {
        p.ei.push_back(edges[2 * k]);
        p.ej.push_back(edges[2 * k + 1]);
        p.J.push_back(J[k]);
    }
    p.h2.assign(n, 0);
    if (h2) for (int i = 0; i < n; i++) p.h2[i] = h2[i];
    return load_common(ctx, std::move(p));
}

int bbtn_load_mwis(bbtn_ctx *ctx, int n, int m, const int32_t *edges, const int32_t *w) {
    if (!ctx || n < 1 || m < 0 || (m > 0 && !edges)) {
        set_error("bad arguments to bbtn_load_mwis");
        return BBTN_EINVAL;
    }
    Problem p;
    p.kind = kMwis;
    p.n = n;
    for (int k = 0; k < m; k++) {
        p.ei.push_back(edges[2 * k]);
        p.ej.push_back(edges[2 * k + 1]);
    }
    p.w.assign(n, 1);
    if (w) for (int i = 0; i < n; i++) p.w[i] = w[i];
    return load_common(ctx, std::move(p));
}

int bbtn_load_file(bbtn_ctx *ctx, const char *path) {
    return guarded([&] {
        if (!ctx || !path) fail(BBTN_EINVAL, "bad arguments");
        ctx->shard.reset();
        ctx->prob = read_problem_file(path);
        ctx->loaded = true;
        ctx->solved = false;
    });
}

int bbtn_solve(bbtn_ctx *ctx, int want_count, int want_config) {
    return guarded([&] {
        if (!ctx) fail(BBTN_EINVAL, "ctx is NULL");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        ctx->solved = false;
        ctx->shard.reset();   // so is any other solve on the context
        if (ctx->device < 0) fail(BBTN_ECUDA, "no CUDA device available");
        BBTN_CUDA(cudaSetDevice(ctx->device));
        Solver s(ctx->opts, ctx->stream, &ctx->arena, &ctx->tuner);
        s.set_gnn(ctx->gnn_branch, ctx->gnn_value);
        ctx->out = s.solve(ctx->prob, want_count != 0, want_config != 0, &ctx->stats);
        ctx->solved = true;
        if (ctx->out.checked) {
            // the residues after the CRT ones are those of the check plane
            std::vector<uint64_t> r(ctx->out.res.begin(), ctx->out.res.begin() + ctx->out.n_crt);
            std::vector<uint64_t> p(ctx->out.primes.begin(), ctx->out.primes.begin() + ctx->out.n_crt);
            for (size_t u = ctx->out.n_crt; u < ctx->out.res.size(); u++)
                if (crt_mod(r, p, ctx->out.primes[u]) != ctx->out.res[u])
                    fail(BBTN_EOVERFLOW, "degeneracy exceeds the range of the CRT primes; use more primes");
        }
    });
}

int bbtn_shard_values(bbtn_ctx *ctx, int rank, int world, int want_count, int64_t *local_max) {
    return guarded([&] {
        if (!ctx || !local_max) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        if (world < 1 || rank < 0 || rank >= world) fail(BBTN_EINVAL, "rank outside 0..world-1");
        if (ctx->opts.mode != BBTN_MODE_BBTN) fail(BBTN_EINVAL, "branch sharding needs BBTN mode");
        if (ctx->device < 0) fail(BBTN_ECUDA, "no CUDA device available");
        BBTN_CUDA(cudaSetDevice(ctx->device));
        ctx->solved = false;
        ctx->shard.reset(new Solver(ctx->opts, ctx->stream, &ctx->arena, &ctx->tuner));
        ctx->shard->set_gnn(ctx->gnn_branch, ctx->gnn_value);
        try {
            *local_max = ctx->shard->shard_values(ctx->prob, rank, world, want_count != 0, &ctx->stats);
        } catch (...) {
            ctx->shard.reset();
            throw;
        }
    });
}

int bbtn_shard_counts(bbtn_ctx *ctx, int64_t global_max, int want_config, int32_t *value, uint64_t *planes,
                      uint64_t *moduli, int *np, int *n_crt_planes, int8_t *config, int *have_config) {
    return guarded([&] {
        if (!ctx || !value || !np || !n_crt_planes) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->shard) fail(BBTN_ESTATE, "bbtn_shard_values has not run on this context");
        if (want_config && (!config || !have_config)) fail(BBTN_EINVAL, "config output missing");
        BBTN_CUDA(cudaSetDevice(ctx->device));
        Solver::ShardResult r;
        try {
            r = ctx->shard->shard_counts(global_max, want_config != 0);
        } catch (...) {
            ctx->shard.reset();
            throw;
        }
        ctx->shard.reset();
        *value = r.value;
        *np = (int)r.planes.size();
        *n_crt_planes = r.n_crt_planes;
        for (size_t t = 0; t < r.planes.size(); t++) {
            if (planes) planes[t] = r.planes[t];
            if (moduli) moduli[t] = r.moduli[t];
        }
        if (have_config) *have_config = r.have_x ? 1 : 0;
        if (r.have_x && config)
            for (size_t i = 0; i < r.x.size(); i++) config[i] = ctx->prob.kind == kSpin ? (int8_t)(2 * r.x[i] - 1) : r.x[i];
    });
}

int bbtn_count_decimal(int np, int n_crt_planes, const uint64_t *planes, const uint64_t *moduli, char *buf,
                       size_t cap, size_t *needed) {
    return guarded([&] {
        if (np < 1 || np > kMaxPlanes || n_crt_planes < 1 || n_crt_planes > np || !planes || !moduli)
            fail(BBTN_EINVAL, "bad count planes");
        uint32_t c[kMaxPlanes];
        plane_moduli(np, moduli, c);   // checks the moduli
        std::vector<uint64_t> r, p;
        for (int t = 0; t < np; t++) {
            if (is_pair(c[t])) {
                const uint64_t q0 = moduli[t] & 0xffffffffull, q1 = moduli[t] >> 32;
                const uint64_t lo = planes[t] & 0xffffffffull, hi = planes[t] >> 32;
                if (lo >= q0 || hi >= q1) fail(BBTN_EINVAL, "residue not below its modulus");
                r.push_back(lo);
                p.push_back(q0);
                r.push_back(hi);
                p.push_back(q1);
            } else {
                if (planes[t] >= moduli[t]) fail(BBTN_EINVAL, "residue not below its modulus");
                r.push_back(planes[t]);
                p.push_back(moduli[t]);
            }
        }
        const size_t k = is_pair(c[0]) ? 2 * (size_t)n_crt_planes : (size_t)n_crt_planes;
        std::vector<uint64_t> rk(r.begin(), r.begin() + k), pk(p.begin(), p.begin() + k);
        for (size_t u = k; u < r.size(); u++)
            if (crt_mod(rk, pk, p[u]) != r[u])
                fail(BBTN_EOVERFLOW, "degeneracy exceeds the range of the CRT primes; use more primes");
        std::string s = crt_decimal(rk, pk);
        if (needed) *needed = s.size() + 1;
        if (buf) {
            if (cap < s.size() + 1) fail(BBTN_EINVAL, "buffer too small");
            memcpy(buf, s.c_str(), s.size() + 1);
        }
    });
}

int bbtn_get_energy(bbtn_ctx *ctx, int64_t *e) {
    return guarded([&] {
        if (!ctx || !e) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->solved) fail(BBTN_ESTATE, "not solved");
        // max-plus value of -2H (spin) -> 2H*; MWIS value is alpha itself
        *e = ctx->prob.kind == kSpin ? -ctx->out.value : ctx->out.value;
    });
}

int bbtn_get_count_residues(bbtn_ctx *ctx, uint64_t *res, uint64_t *primes, int *k) {
    return guarded([&] {
        if (!ctx || !k) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->solved) fail(BBTN_ESTATE, "not solved");
        *k = ctx->out.n_crt;
        for (int t = 0; t < ctx->out.n_crt; t++) {
            if (res) res[t] = ctx->out.res[t];
            if (primes) primes[t] = ctx->out.primes[t];
        }
    });
}

int bbtn_get_count_dec(bbtn_ctx *ctx, char *buf, size_t cap, size_t *needed) {
    return guarded([&] {
        if (!ctx) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->solved) fail(BBTN_ESTATE, "not solved");
        if (ctx->out.n_crt == 0) fail(BBTN_ESTATE, "counts were not requested");
        std::vector<uint64_t> r(ctx->out.res.begin(), ctx->out.res.begin() + ctx->out.n_crt);
        std::vector<uint64_t> p(ctx->out.primes.begin(), ctx->out.primes.begin() + ctx->out.n_crt);
        std::string s = crt_decimal(r, p);
        if (needed) *needed = s.size() + 1;
        if (buf) {
            if (cap < s.size() + 1) fail(BBTN_EINVAL, "buffer too small");
            memcpy(buf, s.c_str(), s.size() + 1);
        }
    });
}

int bbtn_get_config(bbtn_ctx *ctx, int8_t *s) {
    return guarded([&] {
        if (!ctx || !s) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->solved || !ctx->out.have_x) fail(BBTN_ESTATE, "no configuration (solve with want_config)");
        for (int i = 0; i < ctx->prob.n; i++)
            s[i] = ctx->prob.kind == kSpin ? (int8_t)(2 * ctx->out.x[i] - 1) : ctx->out.x[i];
    });
}

int bbtn_analyze(bbtn_ctx *ctx, bbtn_plan_info *info, const char *dump_path) {
    return guarded([&] {
        if (!ctx || !info) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        Solver s(ctx->opts, ctx->stream, &ctx->arena);
        s.set_gnn(ctx->gnn_branch, nullptr);   // a branch scorer runs on the device
        s.analyze(ctx->prob, info, dump_path);
    });
}

int bbtn_get_stats(bbtn_ctx *ctx, bbtn_stats *st) {
    return guarded([&] {
        if (!ctx || !st) fail(BBTN_EINVAL, "bad arguments");
        *st = ctx->stats;
    });
}

}  // extern "C"

// ------------------------------------------------------------ learned branching (GNN)

struct bbtn_gnn {
    std::unique_ptr<GnnModel> m;
    cudaStream_t stream = nullptr;
};

namespace {

void edge_lists(int n, int m, const int32_t *edges, std::vector<int> &ei, std::vector<int> &ej) {
    if (n < 0 || m < 0 || (m > 0 && !edges)) fail(BBTN_EINVAL, "bad graph");
    ei.resize(m);
    ej.resize(m);
    for (int k = 0; k < m; k++) {
        ei[k] = edges[2 * k];
        ej[k] = edges[2 * k + 1];
        if (ei[k] < 0 || ei[k] >= n || ej[k] < 0 || ej[k] >= n || ei[k] == ej[k])
            fail(BBTN_EINVAL, "edge endpoint out of range or self-loop");
    }
}

bbtn_gnn *gnn_checked(bbtn_gnn *g) {
    if (!g || !g->m) fail(BBTN_EINVAL, "gnn is NULL");
    return g;
}

}  // namespace

extern "C" {

int bbtn_gnn_create(uint64_t seed, bbtn_gnn **out) {
    return guarded([&] {
        if (!out) fail(BBTN_EINVAL, "out is NULL");
        int dev = -1;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            fail(BBTN_ECUDA, "no CUDA device available");
        }
        auto g = std::make_unique<bbtn_gnn>();
        g->m = std::make_unique<GnnModel>(seed);
        *out = g.release();
    });
}

void bbtn_gnn_destroy(bbtn_gnn *g) { delete g; }

int bbtn_gnn_param_count(void) { return gnn_param_count(); }

int bbtn_gnn_set_stream(bbtn_gnn *g, void *stream) {
    return guarded([&] { gnn_checked(g)->stream = (cudaStream_t)stream; });
}

int bbtn_gnn_features(int n, int m, const int32_t *edges, const int32_t *w, const int8_t *fixed,
                      const float *score, float *out) {
    return guarded([&] {
        if (!out && n > 0) fail(BBTN_EINVAL, "out is NULL");
        std::vector<int> ei, ej;
        edge_lists(n, m, edges, ei, ej);
        std::vector<int32_t> wv(n, 1);
        std::vector<int8_t> fx(n, -1);
        for (int v = 0; v < n; v++) {
            if (w) wv[v] = w[v];
            if (fixed) {
                if (fixed[v] < -1 || fixed[v] > 1) fail(BBTN_EINVAL, "fixed values must be -1, 0 or 1");
                fx[v] = fixed[v];
            }
        }
        std::vector<float> f, sc;
        if (score) sc.assign(score, score + n);
        gnn_features(n, ei, ej, wv, fx, f, score ? &sc : nullptr);
        if (n > 0) memcpy(out, f.data(), f.size() * sizeof(float));
    });
}

int bbtn_gnn_set_graph(bbtn_gnn *g, int n, int m, const int32_t *edges) {
    return guarded([&] {
        gnn_checked(g);
        if (n < 1) fail(BBTN_EINVAL, "graph needs at least one vertex");
        std::vector<int> ei, ej;
        edge_lists(n, m, edges, ei, ej);
        g->m->set_graph(n, ei, ej, g->stream);
    });
}

int bbtn_gnn_forward(bbtn_gnn *g, const float *feats, float *scores) {
    return guarded([&] {
        gnn_checked(g);
        if (g->m->n < 1) fail(BBTN_ESTATE, "no graph set");
        if (!feats || !scores) fail(BBTN_EINVAL, "feats / scores missing");
        std::vector<float> s;
        g->m->forward(feats, s, g->stream);
        memcpy(scores, s.data(), s.size() * sizeof(float));
    });
}

int bbtn_gnn_train_step(bbtn_gnn *g, const float *feats, const float *labels, const float *mask, float lr,
                        float *loss) {
    return guarded([&] {
        gnn_checked(g);
        if (g->m->n < 1) fail(BBTN_ESTATE, "no graph set");
        if (!feats || !labels || !mask) fail(BBTN_EINVAL, "feats / labels / mask missing");
        const float l = g->m->train_step(feats, labels, mask, lr, g->stream);
        if (loss) *loss = l;
    });
}

int bbtn_gnn_get_params(bbtn_gnn *g, float *p) {
    return guarded([&] {
        gnn_checked(g);
        if (!p) fail(BBTN_EINVAL, "p is NULL");
        std::vector<float> v;
        g->m->get_params(v);
        memcpy(p, v.data(), v.size() * sizeof(float));
    });
}

int bbtn_gnn_set_params(bbtn_gnn *g, const float *p) {
    return guarded([&] {
        gnn_checked(g);
        if (!p) fail(BBTN_EINVAL, "p is NULL");
        std::vector<float> v(p, p + gnn_param_count());
        for (float x : v) if (!std::isfinite(x)) fail(BBTN_EINVAL, "non-finite parameter");
        g->m->set_params(v);
    });
}

int bbtn_gnn_get_grads(bbtn_gnn *g, float *grad) {
    return guarded([&] {
        gnn_checked(g);
        if (!grad) fail(BBTN_EINVAL, "grad is NULL");
        std::vector<float> v;
        g->m->get_grads(v);
        memcpy(grad, v.data(), v.size() * sizeof(float));
    });
}

int bbtn_set_gnn(bbtn_ctx *ctx, bbtn_gnn *branch_scorer, bbtn_gnn *value_model) {
    return guarded([&] {
        if (!ctx) fail(BBTN_EINVAL, "ctx is NULL");
        ctx->gnn_branch = branch_scorer ? gnn_checked(branch_scorer)->m.get() : nullptr;
        ctx->gnn_value = value_model ? gnn_checked(value_model)->m.get() : nullptr;
    });
}

int bbtn_branch_samples(bbtn_ctx *ctx, int max_rows, int lookahead, int8_t *fx, float *score, float *gamma,
                        int *rows) {
    return guarded([&] {
        if (!ctx || !rows) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        if (max_rows < 0 || (max_rows > 0 && (!fx || !score || !gamma))) fail(BBTN_EINVAL, "bad row buffers");
        const int n = ctx->prob.n;
        BranchLog log;
        log.max = max_rows;
        log.lookahead = std::max(1, lookahead);
        log.fx.assign((size_t)max_rows * n, -1);
        log.score.assign((size_t)max_rows * n, 0.f);
        log.gamma.assign((size_t)max_rows * n, -1.f);
        bbtn_opts o = ctx->opts;
        o.mode = BBTN_MODE_BBTN;
        Solver s(o, nullptr, &ctx->arena);
        bbtn_stats st;
        s.branch_samples(ctx->prob, &log, &st);
        const size_t cnt = (size_t)log.count * n;
        if (cnt) {
            memcpy(fx, log.fx.data(), cnt);
            memcpy(score, log.score.data(), cnt * sizeof(float));
            memcpy(gamma, log.gamma.data(), cnt * sizeof(float));
        }
        *rows = log.count;
    });
}

int bbtn_clear_order_cache(void) {
    return guarded([&] { clear_order_cache(); });
}

int bbtn_prepare(bbtn_ctx *ctx) {
    return guarded([&] {
        if (!ctx) fail(BBTN_EINVAL, "ctx is NULL");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        Solver s(ctx->opts, nullptr, &ctx->arena);
        bbtn_stats st{};
        s.prepare(ctx->prob, &st);
    });
}

int bbtn_search_leaves(bbtn_ctx *ctx, int64_t max_leaves, int8_t *fx, int64_t *leaves) {
    return guarded([&] {
        if (!ctx || !leaves || max_leaves < 0 || (max_leaves > 0 && !fx)) fail(BBTN_EINVAL, "bad arguments");
        if (!ctx->loaded) fail(BBTN_ESTATE, "no instance loaded");
        bbtn_opts o = ctx->opts;
        o.mode = BBTN_MODE_BBTN;
        Solver s(o, nullptr, &ctx->arena);
        s.set_gnn(ctx->gnn_branch, nullptr);
        bbtn_stats st{};
        std::vector<int8_t> all;
        s.search_leaves(ctx->prob, max_leaves, all, &st);
        if (!all.empty()) memcpy(fx, all.data(), all.size());
        *leaves = st.leaves;
    });
}

}  // extern "C"

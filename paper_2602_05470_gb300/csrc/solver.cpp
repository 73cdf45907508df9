#include "solver.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <unordered_map>
#include <functional>
#include <thread>

#include "common.h"

namespace bbtn {

namespace {

struct Rng {
    uint64_t s;
    explicit Rng(uint64_t seed) : s(seed) {}
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
    uint64_t below(uint64_t n) { return next() % n; }
};

// Largest tensor and Eq. (4) overflow of the reference tree with fixed variables
// removed; `over` receives the overflowing nodes.
struct Overflow {
    int sc = 0;
    double rho = 0;
    std::vector<int> nodes;   // node ids with effective size > cap
    std::vector<int> size;    // their effective sizes
};

Overflow overflow_of(const CTree &t, const std::vector<int8_t> &fx, int cap) {
    Overflow o;
    for (size_t i = 0; i < t.nodes.size(); i++) {
        int s = 0;
        for (int l : t.nodes[i].lab) if (fx[l] < 0) s++;
        o.sc = std::max(o.sc, s);
        if (s > cap) {
            o.rho += s - cap;
            o.nodes.push_back((int)i);
            o.size.push_back(s);
        }
    }
    return o;
}

// One branching step at a node (paper: branching region R, feasible local
// configurations F(R), optimal branching D(R)). R is grown from `seed` by BFS over
// free variables, preferring overflow-carrying ones. Returns gamma of the chosen
// D(R) (0 when F(R) is empty: the node holds no feasible configuration) and the
// clauses as base-3 states over R (digit 0 free, 1 fixed to 0, 2 fixed to 1).
double branch_at(const Problem &p, const CTree &tree, int cap, const std::vector<int8_t> &fx, const Overflow &ov,
                 const std::vector<double> &score, int seed, int K, std::vector<int> &R,
                 std::vector<int> &clause_states) {
    std::vector<int> pow3(K + 1, 1);
    for (int i = 1; i <= K; i++) pow3[i] = pow3[i - 1] * 3;
    R.clear();
    clause_states.clear();
    const auto &tree_ = tree;
    R.push_back(seed);
    std::vector<char> inR(p.n, 0);
    inR[seed] = 1;
    while ((int)R.size() < K) {
        int pick = -1;
        double pk = -1;
        for (int v : R)
            for (auto &nb : p.adj[v]) {
                int u = nb.first;
                if (inR[u] || fx[u] >= 0) continue;
                int links = 0;
                for (auto &nb2 : p.adj[u]) if (inR[nb2.first]) links++;
                double key = score[u] + 0.25 * links;
                if (key > pk) { pk = key; pick = u; }
            }
        if (pick < 0) break;
        R.push_back(pick);
        inR[pick] = 1;
    }
    const int k = (int)R.size();
    // ---- feasible local configurations F(R): boundary equivalence (per boundary
    // state keep every configuration of maximal local value -- ties kept)
    std::vector<int> bpos;    // indices into R of boundary variables
    for (int i = 0; i < k; i++) {
        bool b = false;
        for (auto &nb : p.adj[R[i]]) if (!inR[nb.first] && fx[nb.first] < 0) { b = true; break; }
        if (b) bpos.push_back(i);
    }
    std::vector<int64_t> lval(1u << k);
    std::vector<char> feas(1u << k, 1);
    for (uint32_t c = 0; c < (1u << k); c++) {
        int64_t val = 0;
        for (int i = 0; i < k && feas[c]; i++) {
            const int v = R[i];
            const int xi = (c >> i) & 1;
            if (p.kind == kMwis) {
                if (xi) {
                    val += p.w[v];
                    for (auto &nb : p.adj[v]) {
                        int u = nb.first;
                        if (fx[u] == 1) { feas[c] = 0; break; }
                        if (inR[u]) {
                            int j = (int)(std::find(R.begin(), R.end(), u) - R.begin());
                            if ((c >> j) & 1) { feas[c] = 0; break; }
                        }
                    }
                }
            } else {
                int64_t eff = p.h2[v];
                for (auto &nb : p.adj[v]) {
                    int u = nb.first;
                    if (fx[u] >= 0) eff += 2ll * p.J[nb.second] * (2 * fx[u] - 1);
                    else if (inR[u] && u > v) {
                        int j = (int)(std::find(R.begin(), R.end(), u) - R.begin());
                        const int xj = (int)((c >> j) & 1u);   // signed: 2 * xj - 1 is -1 or +1
                        val += 2ll * p.J[nb.second] * (2 * xi - 1) * (2 * xj - 1);
                    }
                }
                val += eff * (2 * xi - 1);
            }
        }
        lval[c] = val;
    }
    const int nb = (int)bpos.size();
    std::vector<int64_t> bestb(1u << nb, INT64_MIN);
    auto bstate = [&](uint32_t c) {
        uint32_t b = 0;
        for (int q = 0; q < nb; q++) b |= ((c >> bpos[q]) & 1u) << q;
        return b;
    };
    for (uint32_t c = 0; c < (1u << k); c++)
        if (feas[c]) bestb[bstate(c)] = std::max(bestb[bstate(c)], lval[c]);
    if (p.kind == kMwis) {
        // fewer boundary members never constrain the outside more: a strictly
        // better configuration on a subset of the boundary dominates
        for (int q = 0; q < nb; q++)
            for (uint32_t b = 0; b < (1u << nb); b++)
                if ((b >> q) & 1) bestb[b] = std::max(bestb[b], bestb[b ^ (1u << q)]);
    }
    std::vector<uint32_t> F;
    for (uint32_t c = 0; c < (1u << k); c++)
        if (feas[c] && lval[c] == bestb[bstate(c)]) F.push_back(c);
    if (F.empty()) return 0.0;
    // ---- optimal branching D(R): a decision tree over R whose leaves (clauses)
    // are complete and orthogonal by construction; minimise gamma of
    // gamma^rho = sum_i gamma^rho_i (Eq. (4) and the characteristic equation)
    std::vector<uint64_t> nmask(ov.nodes.size(), 0);   // R-bits carried by each overflow node
    std::vector<int> idxR(p.n, -1);
    for (int i = 0; i < k; i++) idxR[R[i]] = i;
    // MWIS: a 1 in R also fixes its free neighbours (outside R too): universe U
    std::vector<int> U(R.begin(), R.end());
    std::vector<int> idxU(p.n, -1);
    for (int i = 0; i < k; i++) idxU[R[i]] = i;
    std::vector<uint64_t> nbmask(k, 0);
    if (p.kind == kMwis) {
        for (int i = 0; i < k; i++)
            for (auto &nbp : p.adj[R[i]]) {
                int u = nbp.first;
                if (fx[u] >= 0) continue;
                if (idxU[u] < 0 && (int)U.size() < 64) { idxU[u] = (int)U.size(); U.push_back(u); }
                if (idxU[u] >= 0) nbmask[i] |= 1ull << idxU[u];
            }
    }
    for (size_t q = 0; q < ov.nodes.size(); q++)
        for (int l : tree_.nodes[ov.nodes[q]].lab)
            if (idxU[l] >= 0 && fx[l] < 0) nmask[q] |= 1ull << idxU[l];
    // overflowing tensors grouped by (R-mask, size): most carry none of U
    double rho_const = 0;
    std::vector<std::pair<std::pair<uint64_t, int>, int>> groups;   // ((mask, size), multiplicity)
    {
        std::vector<std::pair<uint64_t, int>> ms;
        for (size_t q = 0; q < ov.nodes.size(); q++) {
            if (nmask[q] == 0) rho_const += ov.size[q] - cap;
            else ms.push_back({nmask[q], ov.size[q]});
        }
        std::sort(ms.begin(), ms.end());
        for (auto &e : ms) {
            if (!groups.empty() && groups.back().first == e) groups.back().second++;
            else groups.push_back({e, 1});
        }
    }
    const int S = pow3[k];
    std::vector<double> rho(S);
    std::vector<char> cons(S);
    for (int s = 0; s < S; s++) {
        uint64_t fixedm = 0;
        int x = s;
        for (int i = 0; i < k; i++, x /= 3) {
            int d = x % 3;
            if (d) {
                fixedm |= 1ull << i;
                if (d == 2) fixedm |= nbmask[i];
            }
        }
        double r = rho_const;
        for (auto &g : groups) {
            const int sz = g.first.second - __builtin_popcountll(g.first.first & fixedm);
            if (sz > cap) r += (double)(sz - cap) * g.second;
        }
        rho[s] = r;
    }
    // consistent states: some configuration of F(R) agrees with every fixed digit;
    // each c in F marks the 2^k states that fix a subset of R to c's values
    {
        std::vector<int> st(1u << k);
        for (uint32_t c : F) {
            st[0] = 0;
            cons[0] = 1;
            for (uint32_t m = 1; m < (1u << k); m++) {
                const int i = __builtin_ctz(m);
                st[m] = st[m & (m - 1)] + (int)(((c >> i) & 1) + 1) * pow3[i];
                cons[st[m]] = 1;
            }
        }
    }
    const double rho0 = rho[0];
    std::vector<double> memo(S);
    std::vector<int> choice(S);
    // consistent states, most fixed variables first (children before parents)
    static thread_local std::vector<std::vector<int>> by_fixed_k(11);
    std::vector<int> &all = by_fixed_k[k];
    if (all.empty()) {
        std::vector<int> nfix(S);
        for (int s = 0; s < S; s++) {
            int x = s, nf = 0;
            for (int i = 0; i < k; i++, x /= 3) if (x % 3) nf++;
            nfix[s] = nf;
            all.push_back(s);
        }
        std::stable_sort(all.begin(), all.end(), [&](int a, int b) { return nfix[a] > nfix[b]; });
    }
    std::vector<int> by_fixed;
    by_fixed.reserve(S);
    for (int s : all) {
        if (cons[s]) by_fixed.push_back(s);
        else { memo[s] = 0; choice[s] = -1; }
    }
    auto dp = [&](double gamma) {
        const double lg = std::log(gamma);
        for (int s : by_fixed) {
            double best = s == 0 ? INFINITY : std::exp((rho[s] - rho0) * lg);
            int bc = -1;
            int x = s;
            for (int i = 0; i < k; i++, x /= 3) {
                if (x % 3) continue;
                double c = memo[s + pow3[i]] + memo[s + 2 * pow3[i]];
                if (c < best) { best = c; bc = i; }
            }
            memo[s] = best;
            choice[s] = bc;
        }
        return memo[0];
    };
    double lo = 1.0, hi = std::ldexp(1.0, k) + 1;
    for (int it = 0; it < 30; it++) {     // geometric bisection: ln(hi/lo) shrinks to ~5e-9
        double mid = std::sqrt(lo * hi);
        if (dp(mid) <= 1.0) hi = mid; else lo = mid;
    }
    dp(hi);
    std::function<void(int)> collect = [&](int s) {
        if (!cons[s]) return;
        if (choice[s] < 0) { clause_states.push_back(s); return; }
        collect(s + pow3[choice[s]]);
        collect(s + 2 * pow3[choice[s]]);
    };
    collect(0);
    return hi;
}

}  // namespace

namespace {

// f(0..n-1) on up to 16 host threads; the first exception is rethrown here.
void parallel_for(int64_t n, const std::function<void(int64_t)> &f) {
    const int64_t nt = std::min<int64_t>({n, 16, std::max<int64_t>(1, std::thread::hardware_concurrency())});
    if (nt <= 1) {
        for (int64_t i = 0; i < n; i++) f(i);
        return;
    }
    std::vector<std::thread> th;
    std::vector<std::exception_ptr> err(nt);
    for (int64_t t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            try {
                for (int64_t i = t; i < n; i += nt) f(i);
            } catch (...) {
                err[t] = std::current_exception();
            }
        });
    for (auto &x : th) x.join();
    for (auto &e : err)
        if (e) std::rethrow_exception(e);
}

}  // namespace

void Solver::ensure_buffers(int64_t n) {
    // slots 0..n-1 plus one temporary slot at index dcap_; slot 0 (the running
    // counting-sum) survives a reallocation
    if (n <= dcap_) return;
    const int64_t ncap = std::max<int64_t>(n, 64);
    const int planes = std::max(np_, 1);
    int32_t *nv = nullptr;
    uint64_t *nc = nullptr;
    // stream-ordered allocations: no device-wide synchronisation, so solves on
    // other streams keep running
    BBTN_CUDA(cudaMallocAsync(&nv, sizeof(int32_t) * (ncap + 1), stream_));
    BBTN_CUDA(cudaMallocAsync(&nc, sizeof(uint64_t) * planes * (ncap + 1), stream_));
    if (d_val_) {
        BBTN_CUDA(cudaMemcpyAsync(nv, d_val_, sizeof(int32_t), cudaMemcpyDeviceToDevice, stream_));
        for (int t = 0; t < np_; t++)
            BBTN_CUDA(cudaMemcpyAsync(nc + t * (ncap + 1), d_cnt_ + t * (dcap_ + 1), sizeof(uint64_t),
                                      cudaMemcpyDeviceToDevice, stream_));
        BBTN_CUDA(cudaStreamSynchronize(stream_));
    }
    release_buffers();
    d_val_ = nv;
    d_cnt_ = nc;
    dcap_ = ncap;
    scratch_bytes_ = aggregate_scratch_bytes(dcap_ + 1, np_) + 256;
    BBTN_CUDA(cudaMallocAsync(&d_scratch_, scratch_bytes_, stream_));
}

void Solver::release_buffers() {
    if (d_val_) cudaFreeAsync(d_val_, stream_);
    if (d_cnt_) cudaFreeAsync(d_cnt_, stream_);
    if (d_scratch_) cudaFreeAsync(d_scratch_, stream_);
    d_val_ = nullptr;
    d_cnt_ = nullptr;
    d_scratch_ = nullptr;
    dcap_ = 0;
}

namespace {

// Contraction orders already found, by network structure and search settings: a
// second solve (or an earlier host-only analysis, e.g. of the next instance on
// another thread) reuses the tree instead of searching again. Bounded; cleared
// when full.
struct OrderCache {
    std::mutex mu;
    std::unordered_map<uint64_t, CTree> trees;
};
OrderCache &order_cache() {
    static OrderCache c;
    return c;
}

uint64_t order_key(const std::vector<std::vector<int>> &labels, const std::vector<int8_t> &fx, int cap,
                   double w_rho, int trials, int sa_iters, uint64_t seed, bool minfill_odd) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t x) {
        h ^= x + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 1099511628211ull;
    };
    mix(labels.size());
    for (const auto &l : labels) {
        mix(l.size());
        for (int v : l) mix((uint64_t)v);
    }
    mix(fx.size());
    for (int8_t f : fx) mix((uint64_t)(uint8_t)f);
    mix((uint64_t)cap);
    mix((uint64_t)(w_rho * 1024));
    mix((uint64_t)trials);
    mix((uint64_t)sa_iters);
    mix(seed);
    mix((uint64_t)minfill_odd);
    return h;
}

}  // namespace

void clear_order_cache() {
    OrderCache &c = order_cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.trees.clear();
}

// The root order: from the cache when this network (labels of its tensors and
// the root's fixed variables) was ordered before with the same settings.
CTree Solver::cached_order(const std::vector<int8_t> &fx, int cap, double w_rho, int trials, bool minfill_odd) {
    const uint64_t key = order_key(net_.labels, fx, cap, w_rho, trials, opts_.sa_iters, opts_.seed, minfill_odd);
    OrderCache &c = order_cache();
    {
        std::lock_guard<std::mutex> lock(c.mu);
        auto it = c.trees.find(key);
        if (it != c.trees.end()) return it->second;
    }
    CTree t = order_for(fx, cap, w_rho, trials, minfill_odd);
    std::lock_guard<std::mutex> lock(c.mu);
    if (c.trees.size() >= 256) c.trees.clear();
    c.trees[key] = t;
    return t;
}

CTree Solver::order_for(const std::vector<int8_t> &fx, int cap, double w_rho, int trials, bool minfill_odd) {
    std::vector<std::vector<int>> ll(net_.labels.size());
    for (size_t i = 0; i < ll.size(); i++)
        for (int l : net_.labels[i]) if (fx[l] < 0) ll[i].push_back(l);
    return find_order(ll, p_->n, cap, w_rho, trials, opts_.sa_iters, opts_.seed, minfill_odd);
}

// Exact reductions of a partial assignment (logical inference, paper: local
// pruning eliminates provably suboptimal configurations):
//  MWIS  - a vertex set to 1 forces its neighbours to 0;
//        - a free vertex with no free neighbour and no neighbour set to 1 is 1
//          (leaving it out loses w_v > 0 with nothing gained).
//  spin  - a free spin whose neighbours are all fixed takes the sign of its
//          effective field when that field is non-zero (the other sign is
//          strictly worse); with zero field it stays free.
void Solver::simplify(std::vector<int8_t> &fx) const {
    const Problem &p = *p_;
    bool changed = true;
    while (changed) {
        changed = false;
        for (int v = 0; v < p.n; v++) {
            if (p.kind == kMwis) {
                if (fx[v] == 1) {
                    for (auto &nb : p.adj[v])
                        if (fx[nb.first] < 0) { fx[nb.first] = 0; changed = true; }
                } else if (fx[v] < 0) {
                    bool free_nb = false, one_nb = false;
                    for (auto &nb : p.adj[v]) {
                        if (fx[nb.first] < 0) free_nb = true;
                        else if (fx[nb.first] == 1) one_nb = true;
                    }
                    if (one_nb) { fx[v] = 0; changed = true; }
                    else if (!free_nb) { fx[v] = 1; changed = true; }
                }
            } else if (fx[v] < 0) {
                int64_t eff = p.h2[v];
                bool free_nb = false;
                for (auto &nb : p.adj[v]) {
                    if (fx[nb.first] < 0) { free_nb = true; break; }
                    eff += 2ll * p.J[nb.second] * (2 * fx[nb.first] - 1);
                }
                if (!free_nb && eff != 0) { fx[v] = eff > 0 ? 1 : 0; changed = true; }
            }
        }
    }
}

void Solver::setup(const Problem &p, int active_solves, bool want_count) {
    setup_host(p, want_count);
    arena_->stream = stream_;
    // device memory the leaf arenas of one launch group may take: half of what is
    // free, split among the solves running on this device now (each context's arena
    // is its own, so concurrent solves must not each plan for the same free memory)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
        arena_budget_ = (uint64_t)(free_b + (arena_->owned ? arena_->size : 0)) / 2 /
                        (uint64_t)std::max(1, active_solves);
    if (opts_.arena_budget_mb > 0)
        arena_budget_ = std::min<uint64_t>(arena_budget_, (uint64_t)opts_.arena_budget_mb << 20);
    net_.upload(stream_);
    release_buffers();
    ensure_buffers(std::max(opts_.batch, 1) + 1);
    cudaError_t e = launch_fill(d_val_, d_cnt_, 1, (uint64_t)dcap_ + 1, np_, kNeg, 0, stream_);
    if (e != cudaSuccess) fail(BBTN_ECUDA, cudaGetErrorString(e));
}

void Solver::setup_host(const Problem &p, bool want_count) {
    p_ = &p;
    n_crt_ = want_count ? std::max(0, std::min(opts_.n_primes, BBTN_MAX_PRIMES)) : 0;
    if (want_count && n_crt_ == 0) n_crt_ = 1;
    // count planes: by default two residues per word (primes 2^30 - d, 60 bits of range
    // a plane), else one (2^61 - c, 61 bits)
    pair_ = opts_.wide_counts == 0;
    const int bits = pair_ ? 60 : 61;
    check_ = false;
    if (n_crt_ > 0) {
        if (opts_.count_check == 1) check_ = true;
        else if (opts_.count_check < 0) check_ = p.n + 1 > bits * n_crt_ - 2;   // D <= 2^n
    }
    np_ = n_crt_ + (check_ ? 1 : 0);
    primes_.clear();
    if (pair_) {
        const auto &tab = pair_prime_table();
        for (int t = 0; t < np_; t++) {
            const int i = t < n_crt_ ? t : kCheckPrime;
            primes_.push_back(tab[2 * i]);
            primes_.push_back(tab[2 * i + 1]);
            cprime_[t] = kPairFlag | (uint32_t)((1ull << 30) - tab[2 * i]) | (uint32_t)((1ull << 30) - tab[2 * i + 1]) << 10;
        }
    } else {
        const auto &tab = prime_table();
        for (int t = 0; t < n_crt_; t++) primes_.push_back(tab[t]);
        if (check_) primes_.push_back(tab[kCheckPrime]);
        for (int t = 0; t < np_; t++) cprime_[t] = (uint32_t)((1ull << 61) - primes_[t]);
    }

    fx0_.assign(p.n, -1);
    mult_ = 1;
    if (p.kind == kSpin && p.zero_field() && opts_.use_symmetry && p.n > 0) {
        // H(s) = H(-s): fix the highest-degree spin to +1 and double the count
        int best = 0;
        for (int v = 1; v < p.n; v++) if (p.adj[v].size() > p.adj[best].size()) best = v;
        fx0_[best] = 1;
        mult_ = 2;
    }
    simplify(fx0_);

    net_.set_host(build_network(p), p.n);
    const double t0 = now_s();
    const int cap = opts_.space_cap_log2;
    const double w_rho = opts_.mode == BBTN_MODE_PLAIN ? 8.0 : 1.0;
    // root order: four restarts (one from min-fill), or opts.order_restarts with every
    // odd one from min-fill
    if (opts_.order_restarts > 0) tree_ = cached_order(fx0_, cap, w_rho, opts_.order_restarts, true);
    else tree_ = cached_order(fx0_, cap, w_rho, 4);
    Cost c = tree_cost(tree_, cap);
    st_->tc_log2 = c.tc_log2;
    st_->sc_plain_log2 = c.sc;
    st_->t_plan_s += now_s() - t0;
    best_val_ = INT64_MIN;
    incumbent_ = INT64_MIN;
    best_fx_.clear();
    out_ = SolveOutput();
}

// Leaf contractions are enqueued in windows: window_open starts the timing, each
// enqueue plans a list of leaves (host threads) and launches them without waiting
// (leaf i of the list writes its root result to slot s0 + i), and window_close reads
// the values back once. So the host goes on expanding the search tree or planning
// the next leaves while the device contracts the previous ones.
void Solver::window_open() {
    if (win_.open) return;
    BBTN_CUDA(cudaEventCreate(&win_.e0));
    BBTN_CUDA(cudaEventCreate(&win_.e1));
    BBTN_CUDA(cudaEventRecord(win_.e0, stream_));
    win_.tw = now_s();
    win_.rs = RunStats();
    win_.rs.tuner = opts_.autotune ? tuner_ : nullptr;
    win_.rs.prof = opts_.profile ? &prof_ : nullptr;
    if (win_.rs.prof && !prof_.dump && getenv("BBTN_PROFILE_DUMP")) {
        prof_.dump = fopen(getenv("BBTN_PROFILE_DUMP"), "w");
        if (prof_.dump) fprintf(prof_.dump, "ra,rb,rc,rs,ident,bytes,ops,ms,kind,n\n");
    }
    win_.open = true;
}

void Solver::enqueue_leaves(const std::vector<std::vector<int8_t>> &leaves, bool counting, const CTree *tree,
                            int64_t s0) {
    if (leaves.empty()) return;
    const CTree &tr = tree ? *tree : tree_;
    const int64_t n = (int64_t)leaves.size();
    if (s0 + n > dcap_) fail(BBTN_ESTATE, "leaf result slots exhausted");
    const uint64_t plane = (uint64_t)dcap_ + 1;
    // plan every leaf (host threads), then run them in groups that share launches:
    // leaf i of a group gets its own arena at i * stride
    const double tp = now_s();
    std::vector<Plan> plans(n);
    parallel_for(n, [&](int64_t i) {
        plans[i] = make_plan(tr, net_, leaves[i], counting ? np_ : 0, cprime_, false, !opts_.no_chain_fusion);
    });
    st_->t_plan_s += now_s() - tp;
    uint64_t stride = 256;
    for (const Plan &pl : plans) {
        stride = std::max<uint64_t>(stride, (pl.arena_bytes + 255) & ~255ull);
        st_->sc_log2 = std::max(st_->sc_log2, pl.max_rank);
        st_->steps += (int64_t)pl.steps.size();
    }
    const uint64_t budget = !arena_->owned ? arena_->size
                            : opts_.arena_budget_mb > 0 ? arena_budget_
                                                        : std::max<uint64_t>(arena_budget_, arena_->size);
    const int64_t nb = std::max<int64_t>(1, std::min<int64_t>({(int64_t)kBatchMax, (int64_t)(budget / stride), n}));
    arena_->reserve(stride * nb);   // a grown arena replaces the old one in stream order
    for (int64_t i0 = 0; i0 < n; i0 += nb) {
        std::vector<const Plan *> group;
        for (int64_t i = i0; i < std::min(n, i0 + nb); i++) group.push_back(&plans[i]);
        run_plans(group, net_, arena_->ptr, stride, d_val_ + s0 + i0, d_cnt_ + s0 + i0, plane, stream_, &win_.rs,
                  &prog_);
    }
}

// Ends the window: with `aggregate`, slot 0 <- counting-sum of slots 0..n (paper:
// the result is the sum over the branches); returns the values of slots 1..n.
std::vector<int32_t> Solver::window_close(int64_t n, bool aggregate) {
    const uint64_t plane = (uint64_t)dcap_ + 1;
    if (aggregate && n > 0) {
        int32_t *tv = d_val_ + dcap_;            // temporary result slot (last entry)
        uint64_t *tc = d_cnt_ + dcap_;
        cudaError_t e = launch_aggregate(n + 1, d_val_, d_cnt_, plane, np_, cprime_, tv, tc, plane, d_scratch_,
                                         stream_);
        if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("aggregate: ") + cudaGetErrorString(e));
        win_.rs.launches += n + 1 > 256 ? 2 : 1;
        BBTN_CUDA(cudaMemcpyAsync(d_val_, tv, sizeof(int32_t), cudaMemcpyDeviceToDevice, stream_));
        for (int t = 0; t < np_; t++)
            BBTN_CUDA(cudaMemcpyAsync(d_cnt_ + t * plane, tc + t * plane, sizeof(uint64_t),
                                      cudaMemcpyDeviceToDevice, stream_));
    }
    std::vector<int32_t> vals(n);
    if (n > 0)
        BBTN_CUDA(cudaMemcpyAsync(vals.data(), d_val_ + 1, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, stream_));
    BBTN_CUDA(cudaEventRecord(win_.e1, stream_));
    BBTN_CUDA(cudaStreamSynchronize(stream_));
    float ms = 0;
    BBTN_CUDA(cudaEventElapsedTime(&ms, win_.e0, win_.e1));
    cudaEventDestroy(win_.e0);
    cudaEventDestroy(win_.e1);
    win_.open = false;
    RunStats &rs = win_.rs;
    if (rs.prof) {
        prof_.collect();
        st_->prof_ms = prof_.ms;
        st_->prof_bytes = prof_.bytes;
        st_->prof_ops = prof_.ops;
        st_->prof_launches = prof_.launches;
        st_->prof_scount_ms = prof_.scount_ms;
        st_->prof_scount_bytes = prof_.scount_bytes;
        st_->prof_scount_launches = prof_.scount_launches;
        st_->prof_stream_ms = prof_.stream_ms;
        st_->prof_stream_bytes = prof_.stream_bytes;
        st_->prof_stream_launches = prof_.stream_launches;
        st_->prof_tiled_ms = prof_.tiled_ms;
        st_->prof_tiled_ops = prof_.tiled_ops;
        st_->prof_tiled_launches = prof_.tiled_launches;
        st_->prof_tiled16_launches = prof_.tiled16_launches;
        st_->prof_tcount_ms = prof_.tcount_ms;
        st_->prof_tcount_ops = prof_.tcount_ops;
        st_->prof_tcount_bytes = prof_.tcount_bytes;
        st_->prof_tiled_bytes = prof_.tiled_bytes;
        st_->prof_tcount_launches = prof_.tcount_launches;
        st_->prof_chain_ms = prof_.chain_ms;
        st_->prof_chain_bytes = prof_.chain_bytes;
        st_->prof_chain_launches = prof_.chain_launches;
    }
    st_->chains += rs.chains;
    st_->chained_steps += rs.chained_steps;
    st_->kernel_ms += ms;
    st_->t_device_s += now_s() - win_.tw;
    st_->launches += rs.launches;
    st_->tropical_ops += rs.ops;
    st_->bytes_moved += rs.bytes;
    return vals;
}

// The best leaf and the incumbent after a window's values came back.
void Solver::note_leaf_values(const std::vector<std::vector<int8_t>> &leaves, const std::vector<int32_t> &vals) {
    for (size_t i = 0; i < vals.size(); i++) {
        if (vals[i] >= kFiniteMin && vals[i] > best_val_) {
            best_val_ = vals[i];
            best_fx_ = leaves[i];
        }
        incumbent_ = std::max<int64_t>(incumbent_, vals[i] >= kFiniteMin ? vals[i] : INT64_MIN);
    }
}

// Contract a list of leaf sub-networks and wait (each a full contraction of the
// network with its fixed variables sliced out). With counting, fold the results
// into the running counting-sum in slot 0; without, only the leaves' maxima are
// computed (value planes only). Returns the leaves' values.
std::vector<int32_t> Solver::contract_leaves(const std::vector<std::vector<int8_t>> &leaves, bool counting,
                                             const CTree *tree) {
    if (leaves.empty()) return {};
    const int64_t n = (int64_t)leaves.size();
    ensure_buffers(n + 1);   // slots 0..n, temporary at dcap_ > n
    window_open();
    enqueue_leaves(leaves, counting, tree, 1);
    std::vector<int32_t> vals = window_close(n, counting);
    if (counting) st_->leaves += n;
    note_leaf_values(leaves, vals);
    return vals;
}

void Solver::run_plain() {
    Overflow o = overflow_of(tree_, fx0_, opts_.space_cap_log2);
    if (o.sc > opts_.space_cap_log2)
        fail(BBTN_ENOMEM, "plain contraction needs 2^" + std::to_string(o.sc) +
                              " elements, above the space cap 2^" + std::to_string(opts_.space_cap_log2));
    contract_leaves({fx0_});
}

void Solver::run_sliced() {
    const double t0 = now_s();
    CTree t = tree_;
    std::vector<int> vf = dynamic_slicing(t, opts_.space_cap_log2, std::max(1, opts_.sa_iters / 2), opts_.seed);
    tree_ = t;
    st_->t_plan_s += now_s() - t0;
    st_->slices_log2 = (int)vf.size();
    const int max_log2 = opts_.max_slices_log2 > 0 ? opts_.max_slices_log2 : 30;
    if ((int)vf.size() > max_log2)
        fail(BBTN_ENOMEM, "slicing needs 2^" + std::to_string(vf.size()) + " slices");
    uint64_t ns = 1ull << vf.size();
    if (opts_.slice_sample > 0) ns = std::min<uint64_t>(ns, (uint64_t)opts_.slice_sample);   // timing only
    st_->slices_run = (int64_t)ns;
    const int64_t bs = std::max(1, opts_.batch);
    std::vector<std::vector<int8_t>> batch;
    for (uint64_t x = 0; x < ns; x++) {
        std::vector<int8_t> fx = fx0_;
        for (size_t j = 0; j < vf.size(); j++) fx[vf[j]] = (int8_t)((x >> j) & 1);
        batch.push_back(std::move(fx));
        if ((int64_t)batch.size() == bs || x + 1 == ns) {
            contract_leaves(batch);
            batch.clear();
        }
    }
}

int64_t Solver::incumbent_heuristic() {
    const Problem &p = *p_;
    Rng rng(opts_.seed * 31 + 7);
    int64_t best = INT64_MIN;
    if (p.kind == kMwis) {
        for (int rep = 0; rep < 8; rep++) {
            std::vector<int8_t> x = fx0_;
            std::vector<int> deg(p.n, 0);
            for (int v = 0; v < p.n; v++)
                for (auto &nb : p.adj[v]) if (x[nb.first] < 0) deg[v]++;
            while (true) {
                int pick = -1;
                double bestkey = 1e300;
                for (int v = 0; v < p.n; v++) {
                    if (x[v] >= 0) continue;
                    double key = (double)deg[v] / p.w[v] + (rep ? 0.5 * rng.uniform() : 0.0);
                    if (key < bestkey) { bestkey = key; pick = v; }
                }
                if (pick < 0) break;
                x[pick] = 1;
                for (auto &nb : p.adj[pick]) {
                    int u = nb.first;
                    if (x[u] < 0) {
                        x[u] = 0;
                        for (auto &nb2 : p.adj[u]) deg[nb2.first]--;
                    }
                }
            }
            for (auto &v : x) if (v < 0) v = 0;
            int64_t val = objective(p, x);
            best = std::max(best, val);
        }
    } else {
        for (int rep = 0; rep < 8; rep++) {
            std::vector<int8_t> x(p.n);
            for (int v = 0; v < p.n; v++) x[v] = fx0_[v] >= 0 ? fx0_[v] : (int8_t)(rng.next() & 1);
            // greedy single-spin flips until no flip raises -2H
            bool improved = true;
            while (improved) {
                improved = false;
                for (int v = 0; v < p.n; v++) {
                    if (fx0_[v] >= 0) continue;
                    int64_t field = p.h2[v];
                    for (auto &nb : p.adj[v]) field += 2ll * p.J[nb.second] * (2 * x[nb.first] - 1);
                    int s = 2 * x[v] - 1;
                    if (field * s < 0) { x[v] ^= 1; improved = true; }
                }
            }
            best = std::max(best, objective(p, x));
        }
    }
    return best;
}

// Greedy rounding of the model's logits (largest first, keeping the set
// independent), a few times with perturbed logits; the best set found.
int64_t Solver::incumbent_learned() {
    const Problem &p = *p_;
    std::vector<float> feats;
    gnn_features(p.n, p.ei, p.ej, p.w, fx0_, feats);
    gnn_->set_graph(p.n, p.ei, p.ej, stream_);
    gnn_->forward(feats.data(), logit_, stream_);
    Rng rng(opts_.seed * 131 + 3);
    int64_t best = INT64_MIN;
    std::vector<int> ord(p.n);
    std::vector<float> key(p.n);
    for (int rep = 0; rep < 8; rep++) {
        for (int v = 0; v < p.n; v++) key[v] = logit_[v] + (rep ? (float)(0.5 * rng.uniform()) : 0.f);
        for (int v = 0; v < p.n; v++) ord[v] = v;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return key[a] > key[b]; });
        std::vector<int8_t> x = fx0_;
        for (int v : ord) {
            if (x[v] >= 0) continue;
            x[v] = 1;
            for (auto &nb : p.adj[v]) if (x[nb.first] < 0) x[nb.first] = 0;
        }
        best = std::max(best, objective(p, x));
    }
    return best;
}

void Solver::run_bbtn() {
    // a network that already fits the space cap is its own only leaf: contract it once
    // with counts (the value-only pass would only repeat the same contraction)
    if (overflow_of(tree_, fx0_, opts_.space_cap_log2).sc <= opts_.space_cap_log2) {
        st_->nodes++;
        contract_leaves({fx0_});
        return;
    }
    search(false, nullptr);
}

// The branch-and-bound search over sub-networks. Nodes are expanded depth-first
// (best child last on the stack); a node whose reference-tree overflow is zero is a
// leaf. dry: expand the tree on the host only (leaves are counted, not contracted;
// the incumbent is the heuristic one). log: record, for every expanded node, its
// fixings, the overflow score of each variable and the gamma of the branching
// seeded at each candidate variable (the lookahead labels of the learned scorer).
void Solver::search(bool dry, BranchLog *log) {
    const Problem &p = *p_;
    const int cap = opts_.space_cap_log2;
    const int K = std::max(2, std::min(opts_.region_size, 10));
    incumbent_ = incumbent_heuristic();
    // the learned scorers never prune, so the value and the count do not depend on them
    const bool learned = !dry && opts_.use_gnn && gnn_ && p.kind == kMwis && p.n > 0;
    const bool learned_branch = opts_.use_gnn && gnn_branch_ && p.n > 0 && !log;
    logit_.clear();
    if (learned) {
        const double tg = now_s();
        incumbent_ = std::max(incumbent_, incumbent_learned());
        st_->t_plan_s += now_s() - tg;
    }
    if (learned_branch) gnn_branch_->set_graph(p.n, p.ei, p.ej, stream_);
    const int lookahead = log ? std::max(1, log->lookahead) : std::max(1, opts_.branch_lookahead);
    struct BNode {
        std::vector<int8_t> fx;
        int64_t ub;
    };
    std::vector<BNode> stack;
    stack.push_back({fx0_, upper_bound(p, fx0_)});
    std::vector<std::vector<int8_t>> batch;
    const int bs = std::max(1, opts_.batch);
    std::vector<double> score(p.n);
    std::vector<float> feats, blogit;
    std::vector<int32_t> wv = p.kind == kMwis ? p.w : std::vector<int32_t>(p.n, 0);
    if (p.kind != kMwis)
        for (int v = 0; v < p.n; v++) wv[v] = std::abs(p.h2[v]);

    // Two phases: every leaf is first contracted value-only (its maximum, which also
    // raises the incumbent); only the leaves whose maximum equals the global optimum
    // are contracted again with counts -- the others add nothing to the count.
    std::vector<std::vector<int8_t>> cand;     // leaves that may attain the optimum
    std::vector<int32_t> cand_val;
    // Value-only leaves go to the device in groups of up to kBatchMax as soon as a
    // group is complete, without waiting; their maxima come back once `bs` leaves are
    // in flight or the tree is exhausted (then the incumbent rises and prunes).
    std::vector<std::vector<int8_t>> inflight;
    if (!dry) ensure_buffers(std::max(bs, (int)kBatchMax) + 1);
    auto flush = [&]() {
        if (inflight.empty()) return;
        std::vector<int32_t> v = window_close((int64_t)inflight.size(), np_ == 0);
        if (np_ == 0) st_->leaves += (int64_t)inflight.size();
        note_leaf_values(inflight, v);
        if (np_ > 0) {
            for (size_t i = 0; i < inflight.size(); i++)
                if (v[i] >= kFiniteMin && v[i] >= incumbent_) {
                    cand.push_back(std::move(inflight[i]));
                    cand_val.push_back(v[i]);
                }
        }
        inflight.clear();
    };
    while (!stack.empty() || !batch.empty()) {
        if (stack.empty() || (int)batch.size() >= kBatchMax) {
            if (dry) {
                if (leaf_log_)
                    for (auto &fx : batch) {
                        if ((int64_t)leaf_log_->size() >= leaf_log_max_ * (int64_t)p.n) break;
                        leaf_log_->insert(leaf_log_->end(), fx.begin(), fx.end());
                    }
                st_->leaves += (int64_t)batch.size();
                batch.clear();
                continue;
            }
            if ((int64_t)(inflight.size() + batch.size()) + 1 > dcap_) flush();
            window_open();
            enqueue_leaves(batch, np_ == 0, nullptr, 1 + (int64_t)inflight.size());
            for (auto &fx : batch) inflight.push_back(std::move(fx));
            batch.clear();
            if ((int)inflight.size() >= bs || stack.empty()) flush();
            continue;
        }
        BNode nd = std::move(stack.back());
        stack.pop_back();
        if (nd.ub < incumbent_) { st_->pruned++; continue; }     // global pruning (ties kept)
        st_->nodes++;
        const double tp = now_s();
        Overflow ov = overflow_of(tree_, nd.fx, cap);
        if (ov.sc <= cap) {
            batch.push_back(std::move(nd.fx));
            st_->t_plan_s += now_s() - tp;
            continue;
        }
        // ---- seed of the branching region: by default the variable carried by the
        // most overflow; with a lookahead the one (among the top candidates) whose
        // branching has the smallest gamma; with the learned scorer its top pick
        std::fill(score.begin(), score.end(), 0.0);
        for (size_t q = 0; q < ov.nodes.size(); q++)
            for (int l : tree_.nodes[ov.nodes[q]].lab)
                if (nd.fx[l] < 0) score[l] += ov.size[q] - cap;
        std::vector<int> cands;
        for (int v = 0; v < p.n; v++)
            if (nd.fx[v] < 0 && score[v] > 0) cands.push_back(v);
        if (cands.empty()) fail(BBTN_ESTATE, "no branching variable");
        std::stable_sort(cands.begin(), cands.end(), [&](int a, int b) { return score[a] > score[b]; });
        std::vector<int> R, clause_states;
        double gamma = 0;
        int seed = cands[0];
        if (log && log->count < log->max) {
            // the top candidates with their gamma (the labels); the search follows the lookahead
            const size_t base = (size_t)log->count * p.n;
            double smax = score[cands[0]];
            double gbest = INFINITY;
            for (int v = 0; v < p.n; v++) {
                log->fx[base + v] = nd.fx[v];
                log->score[base + v] = (float)(score[v] / smax);
                log->gamma[base + v] = -1.f;
            }
            for (size_t c = 0; c < cands.size() && c < (size_t)lookahead; c++) {
                std::vector<int> r2, c2;
                const double g = branch_at(p, tree_, cap, nd.fx, ov, score, cands[c], K, r2, c2);
                log->gamma[base + cands[c]] = (float)g;
                if (g > 0 && g < gbest) { gbest = g; seed = cands[c]; }
            }
            log->count++;
        } else if (learned_branch) {
            double smax = score[cands[0]];
            std::vector<float> sc(p.n);
            for (int v = 0; v < p.n; v++) sc[v] = (float)(score[v] / smax);
            gnn_features(p.n, p.ei, p.ej, wv, nd.fx, feats, &sc);
            gnn_branch_->forward(feats.data(), blogit, stream_);
            const size_t m = std::max<size_t>(lookahead, kGnnBranchCandidates);
            for (size_t c = 0; c < cands.size() && c < m; c++)
                if (blogit[cands[c]] > blogit[seed]) seed = cands[c];
        } else if (lookahead > 1) {
            double gbest = INFINITY;
            for (size_t c = 0; c < cands.size() && c < (size_t)lookahead; c++) {
                std::vector<int> r2, c2;
                const double g = branch_at(p, tree_, cap, nd.fx, ov, score, cands[c], K, r2, c2);
                if (g > 0 && g < gbest) { gbest = g; seed = cands[c]; }
            }
        }
        gamma = branch_at(p, tree_, cap, nd.fx, ov, score, seed, K, R, clause_states);
        st_->t_plan_s += now_s() - tp;
        if (gamma == 0) { st_->pruned++; continue; }     // F(R) empty: no feasible configuration
        const int k = (int)R.size();
        // ---- children: fix each clause, propagate, bound
        std::vector<BNode> kids;
        for (int s : clause_states) {
            BNode ch;
            ch.fx = nd.fx;
            int x = s;
            for (int i = 0; i < k; i++, x /= 3)
                if (x % 3) ch.fx[R[i]] = (int8_t)(x % 3 - 1);
            simplify(ch.fx);
            ch.ub = upper_bound(p, ch.fx);
            if (ch.ub < incumbent_) { st_->pruned++; continue; }
            kids.push_back(std::move(ch));
        }
        if (learned) {
            // agreement of each clause with the model: sum of log P(x_v = fixed value)
            // over the variables it fixes; the most likely child is visited first
            std::vector<std::pair<double, size_t>> key(kids.size());
            for (size_t c = 0; c < kids.size(); c++) {
                double a = 0;
                for (int v = 0; v < p.n; v++)
                    if (nd.fx[v] < 0 && kids[c].fx[v] >= 0) {
                        const double z = kids[c].fx[v] ? logit_[v] : -logit_[v];
                        a -= z > 0 ? std::log1p(std::exp(-z)) : -z + std::log1p(std::exp(z));
                    }
                key[c] = {a, c};
            }
            std::stable_sort(key.begin(), key.end());
            std::vector<BNode> sorted;
            for (auto &k2 : key) sorted.push_back(std::move(kids[k2.second]));
            kids.swap(sorted);
        } else {
            std::sort(kids.begin(), kids.end(), [](const BNode &a, const BNode &b) { return a.ub < b.ub; });
        }
        for (auto &ch : kids) stack.push_back(std::move(ch));   // best bound popped first
    }
    flush();   // leaves still in flight when the last nodes were pruned
    if (np_ > 0) {
        std::vector<std::vector<int8_t>> opt;
        for (size_t i = 0; i < cand.size(); i++)
            if (cand_val[i] == incumbent_) opt.push_back(std::move(cand[i]));
        st_->pruned += (int64_t)(cand.size() - opt.size());
        // counting leaves with an order of their own run alone, the others in groups
        // on the root order; each leaf's order is found while the device contracts
        // the previous ones, and the counting-sum waits for all of them once
        for (size_t i0 = 0; i0 < opt.size(); i0 += (size_t)bs) {
            const size_t n = std::min(opt.size() - i0, (size_t)bs);
            ensure_buffers((int64_t)n + 1);
            window_open();
            std::vector<std::vector<int8_t>> rest;
            std::vector<int64_t> rest_slot;
            int64_t slot = 1;
            auto run_rest = [&]() {
                for (size_t j = 0; j < rest.size(); j += kBatchMax) {
                    const size_t m = std::min(rest.size() - j, (size_t)kBatchMax);
                    std::vector<std::vector<int8_t>> g(rest.begin() + j, rest.begin() + j + m);
                    enqueue_leaves(g, true, nullptr, slot);
                    slot += (int64_t)m;
                }
                rest.clear();
            };
            for (size_t i = i0; i < i0 + n; i++) {
                CTree t;
                const double tp = now_s();
                const bool own = leaf_order(opt[i], t);
                st_->t_plan_s += now_s() - tp;
                if (own) enqueue_leaves({opt[i]}, true, &t, slot++);
                else rest.push_back(opt[i]);
                if (rest.size() == (size_t)kBatchMax) run_rest();
            }
            run_rest();
            window_close((int64_t)n, true);
            st_->leaves += (int64_t)n;
        }
    }
}

// A contraction order for one leaf sub-network of its own: opts.leaf_trials greedy +
// annealing runs on the leaf's free variables (one per host thread, different
// seeds). True, with the order in `out`, when the best of them fits the space cap
// with fewer multiply-adds than the root order restricted to the leaf (every
// ordering gives the same contraction value, paper Eq. (2)).
bool Solver::leaf_order(const std::vector<int8_t> &fx, CTree &out) {
    const int trials = opts_.leaf_trials;
    if (trials <= 0) return false;
    const int cap = opts_.space_cap_log2;
    std::vector<char> rem(p_->n, 0);
    for (int v = 0; v < p_->n; v++) rem[v] = fx[v] >= 0;
    const Cost ref = tree_cost(tree_, cap, &rem);
    std::vector<std::vector<int>> ll(net_.labels.size());
    for (size_t i = 0; i < ll.size(); i++)
        for (int l : net_.labels[i]) if (fx[l] < 0) ll[i].push_back(l);
    std::vector<CTree> cand(trials);
    std::vector<Cost> cost(trials);
    parallel_for(trials, [&](int64_t t) {
        cand[t] = find_order(ll, p_->n, cap, 1.0, 1, opts_.sa_iters, opts_.seed * 131 + 17 + (uint64_t)t);
        cost[t] = tree_cost(cand[t], cap);
    });
    int best = -1;
    for (int t = 0; t < trials; t++)
        if (cost[t].sc <= cap && cost[t].tc_log2 < (best < 0 ? ref.tc_log2 : cost[best].tc_log2)) best = t;
    if (best < 0) return false;
    out = std::move(cand[best]);
    return true;
}

void Solver::finish(bool want_config) {
    const uint64_t plane = (uint64_t)dcap_ + 1;
    int32_t v = 0;
    std::vector<uint64_t> r(np_);
    BBTN_CUDA(cudaMemcpyAsync(&v, d_val_, sizeof(int32_t), cudaMemcpyDeviceToHost, stream_));
    for (int t = 0; t < np_; t++)
        BBTN_CUDA(cudaMemcpyAsync(&r[t], d_cnt_ + t * plane, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream_));
    BBTN_CUDA(cudaStreamSynchronize(stream_));
    if (v < kFiniteMin) fail(BBTN_ESTATE, "no feasible configuration");
    out_.value = v;
    if (pair_) {   // one residue per modulus: low half, then high half of each plane
        std::vector<uint64_t> u;
        for (int t = 0; t < np_; t++) {
            u.push_back(r[t] & 0xffffffffull);
            u.push_back(r[t] >> 32);
        }
        r.swap(u);
    }
    for (size_t t = 0; t < r.size(); t++) r[t] = mulmod_host(r[t], mult_ % primes_[t], primes_[t]);
    out_.res = r;
    out_.primes = primes_;
    out_.n_crt = pair_ ? 2 * n_crt_ : n_crt_;
    out_.checked = check_;
    if (want_config) {
        if (best_fx_.empty() || best_val_ != v) fail(BBTN_ESTATE, "optimal branch not recorded");
        // forward with checkpoints and the top-down walk, within the arena budget
        const uint64_t budget =
            opts_.arena_budget_mb > 0 ? (uint64_t)opts_.arena_budget_mb << 20 : arena_budget_;
        const double tp = now_s();
        BackwardPlan bp = make_backward_plan(tree_, net_, best_fx_, budget);
        st_->t_plan_s += now_s() - tp;
        arena_->reserve(bp.arena_bytes);
        int32_t *root = d_val_ + dcap_;
        RunStats rs;
        rs.tuner = opts_.autotune ? tuner_ : nullptr;
        run_backward(bp, tree_, net_, arena_->ptr, root, best_fx_, out_.x, stream_, &rs, &prog_);
        st_->launches += rs.launches;
        st_->bwd_kept = bp.kept;
        st_->bwd_recomputed = bp.recomputed;
        st_->bwd_peak_bytes = bp.peak_bytes;
        st_->bwd_keep_all_bytes = bp.keep_all_bytes;
        st_->bwd_budget_bytes = (double)budget;
        for (auto &xv : out_.x) if (xv < 0) xv = 0;   // variables absent from every tensor
        if (objective(*p_, out_.x) != out_.value)
            fail(BBTN_ESTATE, "recovered configuration does not attain the optimum");
        out_.have_x = true;
    }
}

void Solver::analyze(const Problem &p, bbtn_plan_info *info, const char *dump_path) {
    bbtn_stats st;
    memset(&st, 0, sizeof st);
    st_ = &st;
    setup_host(p, opts_.n_primes > 0);
    memset(info, 0, sizeof(*info));
    Cost c = tree_cost(tree_, opts_.space_cap_log2);
    info->tc_log2 = c.tc_log2;
    info->sc_log2 = c.sc;
    info->rho = c.rho;
    std::vector<int8_t> fx = fx0_;
    if (opts_.mode == BBTN_MODE_SLICED) {
        CTree t = tree_;
        std::vector<int> vf = dynamic_slicing(t, opts_.space_cap_log2, std::max(1, opts_.sa_iters / 2), opts_.seed);
        tree_ = t;
        info->slices_log2 = (int)vf.size();
        for (int v : vf) fx[v] = 0;
    }
    if (opts_.mode == BBTN_MODE_BBTN) {
        search(true, nullptr);
        info->bb_nodes = st.nodes;
        info->bb_leaves = st.leaves;   // the step list below stays that of the root network
        if (c.sc > BBTN_MAX_RANK) return;
    }
    Plan plan = make_plan(tree_, net_, fx, np_, cprime_, false, !opts_.no_chain_fusion);
    info->steps = (int64_t)plan.steps.size();
    info->ops = plan.ops;
    info->bytes = plan.bytes;
    info->arena_bytes = (double)plan.arena_bytes;
    info->chains = (int)plan.chains;
    info->chained_steps = (int)plan.chained_steps;
    {
        const uint64_t budget = opts_.arena_budget_mb > 0 ? (uint64_t)opts_.arena_budget_mb << 20 : 1ull << 30;
        BackwardPlan bp = make_backward_plan(tree_, net_, fx, budget);
        info->bwd_kept = (int)bp.kept;
        info->bwd_recomputed = (int)bp.recomputed;
        info->bwd_peak_bytes = bp.peak_bytes;
        info->bwd_keep_all_bytes = bp.keep_all_bytes;
    }
    if (dump_path) {
        FILE *f = fopen(dump_path, "w");
        if (!f) fail(BBTN_EIO, std::string("cannot write ") + dump_path);
        fprintf(f, "rank_a,rank_b,rank_c,summed,low_identity_bits,bytes,ops,nb,nm,nn,node,a_node,b_node,fused,chain\n");
        for (const PStep &ps : plan.steps) {
            int ra = 0, rb = 0;
            for (int i = 0; i < ps.P.rc; i++) { if (ps.P.oA[i] >= 0) ra++; if (ps.P.oB[i] >= 0) rb++; }
            for (int j = 0; j < ps.P.rs; j++) { if (ps.P.sA[j] >= 0) ra++; if (ps.P.sB[j] >= 0) rb++; }
            int ident = 0;
            while (ident < ps.P.rc && ps.P.oA[ident] == ident && ps.P.oB[ident] < 0) ident++;
            int nb = 0, nm = 0, nn = 0;
            for (int i = 0; i < ps.P.rc; i++) {
                if (ps.P.oA[i] >= 0 && ps.P.oB[i] >= 0) nb++;
                else if (ps.P.oA[i] >= 0) nm++;
                else nn++;
            }
            fprintf(f, "%d,%d,%d,%d,%d,%.0f,%.0f,%d,%d,%d,%d,%d,%d,%d,%d\n", ra, rb, ps.P.rc, ps.P.rs, ident, ps.bytes,
                    ps.ops, nb, nm, nn, ps.node, ps.a_node, ps.b_node, (int)ps.fused, ps.chain_len);
        }
        fclose(f);
    }
}

void Solver::prepare(const Problem &p, bbtn_stats *st) {
    bbtn_stats local{};
    st_ = st ? st : &local;
    setup_host(p, true);
}

void Solver::search_leaves(const Problem &p, int64_t max_leaves, std::vector<int8_t> &fx, bbtn_stats *st) {
    leaf_log_ = &fx;
    leaf_log_max_ = max_leaves;
    fx.clear();
    bbtn_stats local{};
    st_ = st ? st : &local;
    setup_host(p, false);
    search(true, nullptr);
    leaf_log_ = nullptr;
}

int64_t Solver::shard_values(const Problem &p, int rank, int world, bool want_count, bbtn_stats *st) {
    if (world < 1 || rank < 0 || rank >= world) fail(BBTN_EINVAL, "shard: rank outside 0..world-1");
    shard_release();
    st_ = st;
    memset(st, 0, sizeof(*st));
    const double t0 = now_s();
    setup(p, 1, want_count);
    shard_open_ = true;
    // the leaf list of the host-expanded search tree, the same on every rank
    std::vector<int8_t> flat;
    leaf_log_ = &flat;
    leaf_log_max_ = (int64_t)1 << 40;
    const double tp = now_s();
    search(true, nullptr);
    leaf_log_ = nullptr;
    st_->t_plan_s += now_s() - tp;
    const int64_t nleaf = (int64_t)flat.size() / std::max(1, p.n);
    st_->nodes = 0;
    st_->leaves = 0;
    shard_leaves_.clear();
    for (int64_t i = rank; i < nleaf; i += world)
        shard_leaves_.emplace_back(flat.begin() + i * p.n, flat.begin() + (i + 1) * p.n);
    shard_vals_.clear();
    int64_t best = kNeg;
    const int64_t bs = std::max(1, opts_.batch);
    for (size_t i0 = 0; i0 < shard_leaves_.size(); i0 += (size_t)bs) {
        const size_t n = std::min(shard_leaves_.size() - i0, (size_t)bs);
        std::vector<std::vector<int8_t>> g(shard_leaves_.begin() + i0, shard_leaves_.begin() + i0 + n);
        std::vector<int32_t> v = contract_leaves(g, false);
        for (int32_t x : v) {
            shard_vals_.push_back(x);
            if (x >= kFiniteMin) best = std::max<int64_t>(best, x);
        }
    }
    st_->leaves = (int64_t)shard_leaves_.size();
    st_->t_total_s = now_s() - t0;
    return best;
}

Solver::ShardResult Solver::shard_counts(int64_t global_max, bool want_config) {
    if (!shard_open_) fail(BBTN_ESTATE, "shard: values not computed");
    const double t0 = now_s();
    ShardResult r;
    std::vector<std::vector<int8_t>> opt;
    for (size_t i = 0; i < shard_leaves_.size(); i++)
        if (global_max >= kFiniteMin && shard_vals_[i] == global_max) opt.push_back(shard_leaves_[i]);
    const int64_t bs = std::max(1, opts_.batch);
    for (size_t i0 = 0; i0 < opt.size(); i0 += (size_t)bs) {
        const size_t n = std::min(opt.size() - i0, (size_t)bs);
        ensure_buffers((int64_t)n + 1);
        window_open();
        std::vector<std::vector<int8_t>> g(opt.begin() + i0, opt.begin() + i0 + n);
        enqueue_leaves(g, true, nullptr, 1);
        window_close((int64_t)n, true);
    }
    const uint64_t plane = (uint64_t)dcap_ + 1;
    int32_t v = kNeg;
    std::vector<uint64_t> w(np_, 0);
    BBTN_CUDA(cudaMemcpyAsync(&v, d_val_, sizeof(int32_t), cudaMemcpyDeviceToHost, stream_));
    for (int t = 0; t < np_; t++)
        BBTN_CUDA(cudaMemcpyAsync(&w[t], d_cnt_ + t * plane, sizeof(uint64_t), cudaMemcpyDeviceToHost, stream_));
    BBTN_CUDA(cudaStreamSynchronize(stream_));
    if (!opt.empty() && v != global_max) fail(BBTN_ESTATE, "shard: counting pass disagrees with the value pass");
    r.value = opt.empty() ? kNeg : v;
    r.n_crt_planes = n_crt_;
    for (int t = 0; t < np_; t++) {
        uint64_t word = opt.empty() ? 0 : w[t];
        // the spin-flip multiplier, applied per residue like the solver's own result
        if (pair_) {
            const uint64_t q0 = primes_[2 * t], q1 = primes_[2 * t + 1];
            const uint64_t lo = mulmod_host(word & 0xffffffffull, mult_ % q0, q0);
            const uint64_t hi = mulmod_host(word >> 32, mult_ % q1, q1);
            word = lo | hi << 32;
            r.moduli.push_back(q0 | q1 << 32);
        } else {
            word = mulmod_host(word, mult_ % primes_[t], primes_[t]);
            r.moduli.push_back(primes_[t]);
        }
        r.planes.push_back(word);
    }
    st_->leaves += (int64_t)opt.size();
    if (want_config && !opt.empty()) {
        best_fx_ = opt[0];
        best_val_ = global_max;
        finish(true);
        r.x = out_.x;
        r.have_x = true;
    }
    st_->t_total_s += now_s() - t0;
    shard_release();
    return r;
}

void Solver::shard_release() {
    if (!shard_open_) return;
    release_buffers();
    net_.release(stream_);
    shard_leaves_.clear();
    shard_vals_.clear();
    shard_open_ = false;
}

void Solver::branch_samples(const Problem &p, BranchLog *log, bbtn_stats *st) {
    st_ = st;
    memset(st, 0, sizeof(*st));
    setup_host(p, false);
    search(true, log);
}

namespace {

// Solves in progress per device, so that concurrent contexts split the free device
// memory between their arenas instead of each planning for all of it.
struct ActiveSolves {
    std::mutex mu;
    std::unordered_map<int, int> n;
};
ActiveSolves &active_solves() {
    static ActiveSolves a;
    return a;
}
struct ActiveSolve {
    int dev = -1, count = 1;
    ActiveSolve() {
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            dev = -1;
        }
        ActiveSolves &a = active_solves();
        std::lock_guard<std::mutex> lock(a.mu);
        count = ++a.n[dev];
    }
    ~ActiveSolve() {
        ActiveSolves &a = active_solves();
        std::lock_guard<std::mutex> lock(a.mu);
        --a.n[dev];
    }
};

}  // namespace

SolveOutput Solver::solve(const Problem &p, bool want_count, bool want_config, bbtn_stats *st) {
    const double t0 = now_s();
    st_ = st;
    memset(st, 0, sizeof(*st));
    ActiveSolve active;
    try {
        setup(p, active.count, want_count);
        switch (opts_.mode) {
            case BBTN_MODE_PLAIN: run_plain(); break;
            case BBTN_MODE_SLICED: run_sliced(); break;
            default: run_bbtn(); break;
        }
        finish(want_config);
    } catch (...) {
        release_buffers();
        net_.release(stream_);
        throw;
    }
    release_buffers();
    net_.release(stream_);
    st->t_total_s = now_s() - t0;
    return out_;
}

}  // namespace bbtn

#include "order.h"

#include <algorithm>
#include <cmath>
#include <exception>
#include <thread>
#include <limits>
#include <queue>
#include <unordered_set>

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

int union_size(const std::vector<int> &a, const std::vector<int> &b) {
    size_t i = 0, j = 0;
    int n = 0;
    while (i < a.size() && j < b.size()) {
        if (a[i] < b[j]) i++;
        else if (b[j] < a[i]) j++;
        else { i++; j++; }
        n++;
    }
    return n + (int)(a.size() - i) + (int)(b.size() - j);
}

void set_union(const std::vector<int> &a, const std::vector<int> &b, std::vector<int> &out) {
    out.clear();
    std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
}

void set_inter(const std::vector<int> &a, const std::vector<int> &b, std::vector<int> &out) {
    out.clear();
    std::set_intersection(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
}

bool contains(const std::vector<int> &a, int x) { return std::binary_search(a.begin(), a.end(), x); }

double pow2(int k) { return std::ldexp(1.0, k); }

}  // namespace

void recompute_labels(CTree &t) {
    // (label, occurrences in the subtree) merged bottom-up; a label whose count
    // reaches its total has no leaf outside the subtree and is summed there.
    int maxlab = -1;
    for (int i = 0; i < t.nleaves; i++)
        for (int l : t.nodes[i].lab) maxlab = std::max(maxlab, l);
    std::vector<int> total(maxlab + 2, 0);
    for (int i = 0; i < t.nleaves; i++)
        for (int l : t.nodes[i].lab) total[l]++;
    std::vector<std::vector<std::pair<int, int>>> cnt(t.nodes.size());
    std::vector<int> order;
    order.reserve(t.nodes.size());
    // iterative post-order
    std::vector<std::pair<int, int>> st;
    st.push_back({t.root, 0});
    while (!st.empty()) {
        auto &top = st.back();
        const CNode &nd = t.nodes[top.first];
        if (nd.is_leaf() || top.second == 2) {
            order.push_back(top.first);
            st.pop_back();
            continue;
        }
        int child = top.second == 0 ? nd.l : nd.r;
        top.second++;
        st.push_back({child, 0});
    }
    for (int id : order) {
        CNode &nd = t.nodes[id];
        auto &c = cnt[id];
        if (nd.is_leaf()) {
            c.clear();
            for (int l : nd.lab) c.push_back({l, 1});
            continue;
        }
        auto &a = cnt[nd.l], &b = cnt[nd.r];
        c.clear();
        size_t i = 0, j = 0;
        while (i < a.size() || j < b.size()) {
            std::pair<int, int> x;
            if (j >= b.size() || (i < a.size() && a[i].first < b[j].first)) x = a[i++];
            else if (i >= a.size() || b[j].first < a[i].first) x = b[j++];
            else { x = {a[i].first, a[i].second + b[j].second}; i++; j++; }
            if (x.second < total[x.first]) c.push_back(x);
        }
        nd.lab.clear();
        for (auto &x : c) nd.lab.push_back(x.first);
        a.clear(); a.shrink_to_fit();
        b.clear(); b.shrink_to_fit();
    }
}

Cost tree_cost(const CTree &t, int cap, const std::vector<char> *removed) {
    Cost c;
    double tc = 0;
    auto eff = [&](const std::vector<int> &lab) {
        if (!removed) return (int)lab.size();
        int k = 0;
        for (int l : lab) if (!(*removed)[l]) k++;
        return k;
    };
    std::vector<int> u;
    for (size_t i = 0; i < t.nodes.size(); i++) {
        const CNode &nd = t.nodes[i];
        int s = eff(nd.lab);
        c.sc = std::max(c.sc, s);
        if (s > cap) c.rho += s - cap;
        if (!nd.is_leaf()) {
            set_union(t.nodes[nd.l].lab, t.nodes[nd.r].lab, u);
            tc += pow2(eff(u));
        }
    }
    c.tc_log2 = tc > 0 ? std::log2(tc) : 0;
    return c;
}

CTree greedy_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, uint64_t seed,
                   double noise) {
    Rng rng(seed);
    CTree t;
    const int T = (int)leaf_labels.size();
    t.nleaves = T;
    t.nodes.resize(T);
    for (int i = 0; i < T; i++) {
        t.nodes[i].leaf = i;
        t.nodes[i].lab = leaf_labels[i];
        std::sort(t.nodes[i].lab.begin(), t.nodes[i].lab.end());
    }
    if (T == 0) fail(BBTN_EINVAL, "empty network");
    if (T == 1) { t.root = 0; return t; }
    std::vector<int> count(nvars, 0);
    std::vector<std::vector<int>> holders(nvars);
    std::vector<char> alive(2 * T, 0);
    for (int i = 0; i < T; i++) {
        alive[i] = 1;
        for (int l : t.nodes[i].lab) { count[l]++; holders[l].push_back(i); }
    }
    struct Cand { double cost; int a, b; };
    auto cmp = [](const Cand &x, const Cand &y) { return x.cost > y.cost; };
    std::priority_queue<Cand, std::vector<Cand>, decltype(cmp)> pq(cmp);
    std::vector<int> tmp;
    auto out_size = [&](int a, int b) {
        const auto &A = t.nodes[a].lab, &B = t.nodes[b].lab;
        size_t i = 0, j = 0;
        int n = 0;
        while (i < A.size() || j < B.size()) {
            int l, inside;
            if (j >= B.size() || (i < A.size() && A[i] < B[j])) { l = A[i++]; inside = 1; }
            else if (i >= A.size() || B[j] < A[i]) { l = B[j++]; inside = 1; }
            else { l = A[i]; i++; j++; inside = 2; }
            if (count[l] > inside) n++;
        }
        return n;
    };
    auto push = [&](int a, int b) {
        int so = out_size(a, b);
        double cost = pow2(so) - pow2((int)t.nodes[a].lab.size()) - pow2((int)t.nodes[b].lab.size());
        if (noise > 0) cost -= noise * std::log(-std::log(rng.uniform() + 1e-300)) *
                              std::max(1.0, std::fabs(cost));
        pq.push({cost, a, b});
    };
    for (int l = 0; l < nvars; l++) {
        auto &h = holders[l];
        for (size_t i = 0; i < h.size(); i++)
            for (size_t j = i + 1; j < h.size(); j++) push(h[i], h[j]);
    }
    int nalive = T;
    auto merge = [&](int a, int b) {
        CNode nd;
        nd.l = a;
        nd.r = b;
        const auto &A = t.nodes[a].lab, &B = t.nodes[b].lab;
        size_t i = 0, j = 0;
        std::vector<int> all;
        while (i < A.size() || j < B.size()) {
            int l, inside;
            if (j >= B.size() || (i < A.size() && A[i] < B[j])) { l = A[i++]; inside = 1; }
            else if (i >= A.size() || B[j] < A[i]) { l = B[j++]; inside = 1; }
            else { l = A[i]; i++; j++; inside = 2; }
            count[l] -= inside;
            if (count[l] > 0) { nd.lab.push_back(l); count[l]++; }
        }
        int id = (int)t.nodes.size();
        t.nodes[a].parent = id;
        t.nodes[b].parent = id;
        t.nodes.push_back(nd);
        alive[a] = alive[b] = 0;
        alive[id] = 1;
        nalive--;
        std::unordered_set<int> nbrs;
        for (int l : t.nodes[id].lab) {
            auto &h = holders[l];
            size_t w = 0;
            for (size_t k = 0; k < h.size(); k++)
                if (alive[h[k]]) h[w++] = h[k];
            h.resize(w);
            for (int d : h) nbrs.insert(d);
            h.push_back(id);
        }
        for (int d : nbrs) push(id, d);
        return id;
    };
    while (nalive > 1 && !pq.empty()) {
        Cand c = pq.top();
        pq.pop();
        if (!alive[c.a] || !alive[c.b]) continue;
        merge(c.a, c.b);
    }
    if (nalive > 1) {
        // disconnected parts: combine the remaining (label-disjoint) tensors, smallest first
        std::vector<int> rest;
        for (int i = 0; i < (int)t.nodes.size(); i++) if (alive[i]) rest.push_back(i);
        auto bysize = [&](int a, int b) { return t.nodes[a].lab.size() > t.nodes[b].lab.size(); };
        std::priority_queue<int, std::vector<int>, decltype(bysize)> q(bysize);
        for (int x : rest) q.push(x);
        while (q.size() > 1) {
            int a = q.top(); q.pop();
            int b = q.top(); q.pop();
            q.push(merge(a, b));
        }
    }
    for (int i = 0; i < (int)t.nodes.size(); i++) if (alive[i]) t.root = i;
    return t;
}

// Variable elimination order by minimum fill-in: repeatedly eliminate the variable
// whose neighbours in the interaction graph (variables sharing a tensor) need the
// fewest new edges to become a clique, ties broken by degree, then by a seeded
// random key. Its widths on grid-like graphs are close to the sweep widths.
static std::vector<int> min_fill_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, uint64_t seed) {
    Rng rng(seed);
    // the interaction graph as one bit row per variable: a variable's degree is a
    // popcount, its fill (non-adjacent pairs of neighbours) is C(d, 2) minus half the
    // sum over neighbours u of |N(u) & N(v)|, and an elimination ORs the eliminated
    // variable's row into its neighbours' rows
    const int W = (nvars + 63) / 64;
    std::vector<uint64_t> bits((size_t)nvars * W, 0);
    auto row = [&](int v) { return bits.data() + (size_t)v * W; };
    auto set_bit = [&](int v, int w) { row(v)[w >> 6] |= 1ull << (w & 63); };
    std::vector<char> used(nvars, 0);
    for (const auto &lab : leaf_labels)
        for (size_t i = 0; i < lab.size(); i++) {
            used[lab[i]] = 1;
            for (size_t j = i + 1; j < lab.size(); j++) {
                set_bit(lab[i], lab[j]);
                set_bit(lab[j], lab[i]);
            }
        }
    auto degree = [&](int v) {
        const uint64_t *r = row(v);
        int d = 0;
        for (int k = 0; k < W; k++) d += __builtin_popcountll(r[k]);
        return d;
    };
    // calls f(u) for every set bit u of the row r, in ascending order
    auto for_bits = [&](const uint64_t *r, auto &&f) {
        for (int k = 0; k < W; k++)
            for (uint64_t x = r[k]; x; x &= x - 1) f(k * 64 + __builtin_ctzll(x));
    };
    auto fill_of = [&](int v) {
        const uint64_t *rv = row(v);
        int64_t d = 0, adjacent2 = 0;
        for_bits(rv, [&](int u) {
            d++;
            const uint64_t *ru = row(u);
            for (int k = 0; k < W; k++) adjacent2 += __builtin_popcountll(ru[k] & rv[k]);
        });
        return d * (d - 1) / 2 - adjacent2 / 2;
    };
    std::vector<double> tieb(nvars);
    for (int v = 0; v < nvars; v++) tieb[v] = rng.uniform();
    struct Key { int64_t fill; int deg; double r; int v; };
    auto worse = [](const Key &x, const Key &y) {
        if (x.fill != y.fill) return x.fill > y.fill;
        if (x.deg != y.deg) return x.deg > y.deg;
        return x.r > y.r;
    };
    std::priority_queue<Key, std::vector<Key>, decltype(worse)> pq(worse);
    std::vector<int64_t> cur(nvars, -1);
    std::vector<char> gone(nvars, 0);
    for (int v = 0; v < nvars; v++)
        if (used[v]) {
            cur[v] = fill_of(v);
            pq.push({cur[v], degree(v), tieb[v], v});
        }
    std::vector<int> order;
    std::vector<uint64_t> nb(W), touched(W);
    while (!pq.empty()) {
        Key k = pq.top();
        pq.pop();
        const int v = k.v;
        if (gone[v] || k.fill != cur[v] || k.deg != degree(v)) continue;
        gone[v] = 1;
        order.push_back(v);
        // N becomes a clique; v leaves the graph
        std::copy(row(v), row(v) + W, nb.begin());
        for_bits(nb.data(), [&](int a) {
            uint64_t *ra = row(a);
            for (int k2 = 0; k2 < W; k2++) ra[k2] |= nb[k2];
            ra[a >> 6] &= ~(1ull << (a & 63));
            ra[v >> 6] &= ~(1ull << (v & 63));
        });
        std::fill(row(v), row(v) + W, 0ull);
        std::copy(nb.begin(), nb.end(), touched.begin());
        for_bits(nb.data(), [&](int a) {
            const uint64_t *ra = row(a);
            for (int k2 = 0; k2 < W; k2++) touched[k2] |= ra[k2];
        });
        for_bits(touched.data(), [&](int w) {
            if (gone[w]) return;
            cur[w] = fill_of(w);
            pq.push({cur[w], degree(w), tieb[w], w});
        });
    }
    return order;
}

CTree elimination_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, uint64_t seed) {
    const std::vector<int> elim = min_fill_order(leaf_labels, nvars, seed);
    CTree t;
    const int T = (int)leaf_labels.size();
    t.nleaves = T;
    t.nodes.resize(T);
    for (int i = 0; i < T; i++) {
        t.nodes[i].leaf = i;
        t.nodes[i].lab = leaf_labels[i];
        std::sort(t.nodes[i].lab.begin(), t.nodes[i].lab.end());
    }
    if (T == 0) fail(BBTN_EINVAL, "empty network");
    if (T == 1) { t.root = 0; return t; }
    // bucket elimination: all tensors holding the next variable are contracted
    // together (smallest first), so the variable is summed at their last merge
    std::vector<int> count(nvars, 0);
    std::vector<std::vector<int>> holders(nvars);
    std::vector<char> alive(2 * T, 0);
    for (int i = 0; i < T; i++) {
        alive[i] = 1;
        for (int l : t.nodes[i].lab) { count[l]++; holders[l].push_back(i); }
    }
    auto merge = [&](int a, int b) {
        CNode nd;
        nd.l = a;
        nd.r = b;
        const auto &A = t.nodes[a].lab, &B = t.nodes[b].lab;
        size_t i = 0, j = 0;
        while (i < A.size() || j < B.size()) {
            int l, inside;
            if (j >= B.size() || (i < A.size() && A[i] < B[j])) { l = A[i++]; inside = 1; }
            else if (i >= A.size() || B[j] < A[i]) { l = B[j++]; inside = 1; }
            else { l = A[i]; i++; j++; inside = 2; }
            count[l] -= inside;
            if (count[l] > 0) { nd.lab.push_back(l); count[l]++; }
        }
        const int id = (int)t.nodes.size();
        t.nodes[a].parent = id;
        t.nodes[b].parent = id;
        t.nodes.push_back(nd);
        alive[a] = alive[b] = 0;
        alive[id] = 1;
        for (int l : t.nodes[id].lab) holders[l].push_back(id);
        return id;
    };
    auto bysize = [&](int a, int b) { return t.nodes[a].lab.size() > t.nodes[b].lab.size(); };
    for (int v : elim) {
        std::vector<int> S;
        for (int x : holders[v])
            if (alive[x]) S.push_back(x);
        holders[v].clear();
        if (S.size() < 2) {
            for (int x : S) holders[v].push_back(x);
            continue;
        }
        std::priority_queue<int, std::vector<int>, decltype(bysize)> q(bysize);
        for (int x : S) q.push(x);
        while (q.size() > 1) {
            int a = q.top(); q.pop();
            int b = q.top(); q.pop();
            q.push(merge(a, b));
        }
    }
    std::vector<int> rest;
    for (int i = 0; i < (int)t.nodes.size(); i++) if (alive[i]) rest.push_back(i);
    std::priority_queue<int, std::vector<int>, decltype(bysize)> q(bysize);
    for (int x : rest) q.push(x);
    while (q.size() > 1) {
        int a = q.top(); q.pop();
        int b = q.top(); q.pop();
        q.push(merge(a, b));
    }
    t.root = q.top();
    return t;
}

void tree_sa(CTree &t, const SAParams &sp, uint64_t seed) {
    Rng rng(seed);
    std::vector<int> internal;
    for (int i = 0; i < (int)t.nodes.size(); i++)
        if (!t.nodes[i].is_leaf()) internal.push_back(i);
    if (internal.size() < 2) return;
    auto node_cost = [&](int id) {
        const CNode &nd = t.nodes[id];
        return pow2(union_size(t.nodes[nd.l].lab, t.nodes[nd.r].lab));
    };
    auto over = [&](int s) { return s > sp.cap ? (double)(s - sp.cap) : 0.0; };
    double tc = 0, rho = 0;
    for (int id : internal) tc += node_cost(id);
    for (auto &nd : t.nodes) rho += over((int)nd.lab.size());
    std::vector<int> u1, u2, newx;
    const long moves_per = (long)internal.size() * sp.sweeps;
    for (int bs = 0; bs < sp.beta_steps; bs++) {
        const double beta = sp.beta_steps > 1
            ? sp.beta_start + (sp.beta_end - sp.beta_start) * bs / (sp.beta_steps - 1)
            : sp.beta_end;
        for (long mv = 0; mv < moves_per; mv++) {
            const int n = internal[rng.below(internal.size())];
            CNode &N = t.nodes[n];
            const bool lint = !t.nodes[N.l].is_leaf(), rint = !t.nodes[N.r].is_leaf();
            if (!lint && !rint) continue;
            bool pick_left = lint && (!rint || (rng.next() & 1));
            const int x = pick_left ? N.l : N.r;
            const int y = pick_left ? N.r : N.l;
            CNode &X = t.nodes[x];
            const bool gl = rng.next() & 1;
            const int g = gl ? X.l : X.r;     // moves up to n
            const int o = gl ? X.r : X.l;     // stays under x, joined by y
            const auto &Lo = t.nodes[o].lab, &Ly = t.nodes[y].lab, &Lg = t.nodes[g].lab;
            set_union(Lo, Ly, u1);
            set_union(Lg, N.lab, u2);
            set_inter(u1, u2, newx);
            const double old_x = pow2(union_size(t.nodes[X.l].lab, t.nodes[X.r].lab));
            const double old_n = pow2(union_size(X.lab, Ly));
            const double new_x = pow2((int)u1.size());
            const double new_n = pow2(union_size(newx, Lg));
            const double tc_new = tc - old_x - old_n + new_x + new_n;
            const double rho_new = rho - over((int)X.lab.size()) + over((int)newx.size());
            const double f_old = std::log2(tc) + sp.w_rho * rho;
            const double f_new = std::log2(std::max(tc_new, 1.0)) + sp.w_rho * rho_new;
            const double df = f_new - f_old;
            if (df <= 0 || rng.uniform() < std::exp(-beta * df)) {
                X.l = o;
                X.r = y;
                t.nodes[y].parent = x;
                t.nodes[o].parent = x;
                if (pick_left) N.r = g; else N.l = g;
                t.nodes[g].parent = n;
                X.lab = newx;
                tc = tc_new;
                rho = rho_new;
            }
        }
        // re-sum to keep the running total exact
        tc = 0;
        for (int id : internal) tc += node_cost(id);
    }
}

CTree find_order(const std::vector<std::vector<int>> &leaf_labels, int nvars, int cap, double w_rho,
                 int trials, int sa_beta_steps, uint64_t seed, bool minfill_odd) {
    // independent restarts, one host thread each; the best objective wins (ties:
    // the lowest trial index, so the result does not depend on thread timing)
    const int nt = std::max(1, trials);
    std::vector<CTree> trees(nt);
    std::vector<double> f(nt, std::numeric_limits<double>::infinity());
    auto run = [&](int tr) {
        // restart 1 (every odd one with minfill_odd) starts from a min-fill elimination
        // order, the others from greedy
        CTree t = tr == 1 || (minfill_odd && tr % 2 == 1) ? elimination_order(leaf_labels, nvars, seed * 7919 + tr)
                          : greedy_order(leaf_labels, nvars, seed * 7919 + tr, tr == 0 ? 0.0 : 0.3);
        if (sa_beta_steps > 0) {
            SAParams sp;
            sp.cap = cap;
            sp.w_rho = w_rho;
            sp.beta_steps = sa_beta_steps;
            tree_sa(t, sp, seed * 104729 + tr);
        }
        Cost c = tree_cost(t, cap);
        f[tr] = c.tc_log2 + w_rho * c.rho;
        trees[tr] = std::move(t);
    };
    if (nt == 1) {
        run(0);
    } else {
        std::vector<std::thread> th;
        std::vector<std::exception_ptr> err(nt);
        for (int tr = 0; tr < nt; tr++)
            th.emplace_back([&, tr] {
                try {
                    run(tr);
                } catch (...) {
                    err[tr] = std::current_exception();
                }
            });
        for (auto &x : th) x.join();
        for (auto &e : err)
            if (e) std::rethrow_exception(e);
    }
    int best = 0;
    for (int tr = 1; tr < nt; tr++)
        if (f[tr] < f[best]) best = tr;
    return std::move(trees[best]);
}

std::vector<int> dynamic_slicing(CTree &t, int cap, int sa_beta_steps, uint64_t seed) {
    std::vector<int> sliced;
    int maxlab = 0;
    for (auto &nd : t.nodes) for (int l : nd.lab) maxlab = std::max(maxlab, l + 1);
    int round = 0;
    while (true) {
        Cost c = tree_cost(t, cap);
        if (c.sc <= cap) break;
        // candidates: labels of the largest tensors
        std::vector<int> cand;
        for (auto &nd : t.nodes)
            if ((int)nd.lab.size() == c.sc) for (int l : nd.lab) cand.push_back(l);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        int best = -1;
        double best_over = 1e300, best_tc = 1e300;
        std::vector<int> u;
        for (int l : cand) {
            double ov = 0, tc = 0;
            for (auto &nd : t.nodes) {
                int s = (int)nd.lab.size() - (contains(nd.lab, l) ? 1 : 0);
                if (s > cap) ov += pow2(s - cap);
                if (!nd.is_leaf()) {
                    set_union(t.nodes[nd.l].lab, t.nodes[nd.r].lab, u);
                    tc += pow2((int)u.size() - (contains(u, l) ? 1 : 0));
                }
            }
            if (ov < best_over || (ov == best_over && tc < best_tc)) {
                best_over = ov; best_tc = tc; best = l;
            }
        }
        if (best < 0) fail(BBTN_ENOMEM, "slicing found no candidate");
        sliced.push_back(best);
        for (auto &nd : t.nodes) {
            auto it = std::lower_bound(nd.lab.begin(), nd.lab.end(), best);
            if (it != nd.lab.end() && *it == best) nd.lab.erase(it);
        }
        // the tree of one slice may now be improvable: re-anneal every few slices
        if (sa_beta_steps > 0 && (++round % 4) == 0) {
            SAParams sp;
            sp.cap = cap;
            sp.w_rho = 4.0;
            sp.beta_steps = sa_beta_steps;
            sp.beta_start = 5.0;
            tree_sa(t, sp, seed + round);
        }
        if ((int)sliced.size() > 62) fail(BBTN_ENOMEM, "more than 62 sliced variables");
    }
    return sliced;
}

}  // namespace bbtn

#include "network.h"

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <fstream>
#include <set>
#include <sstream>

#include "common.h"
#include "semiring.cuh"

namespace bbtn {

bool Problem::zero_field() const {
    for (auto h : h2) if (h) return false;
    return true;
}

void Problem::build_adjacency() {
    adj.assign(n, {});
    for (int k = 0; k < m(); k++) {
        adj[ei[k]].push_back({ej[k], k});
        adj[ej[k]].push_back({ei[k], k});
    }
}

void validate(Problem &p) {
    if (p.n < 1 || p.n > (1 << 24)) fail(BBTN_EINVAL, "vertex count out of range");
    std::set<std::pair<int, int>> seen;
    for (int k = 0; k < p.m(); k++) {
        int a = p.ei[k], b = p.ej[k];
        if (a < 0 || b < 0 || a >= p.n || b >= p.n) fail(BBTN_EINVAL, "edge endpoint out of range");
        if (a == b) fail(BBTN_EINVAL, "self loop");
        if (a > b) std::swap(a, b);
        if (!seen.insert({a, b}).second) fail(BBTN_EINVAL, "duplicate edge");
        p.ei[k] = a;
        p.ej[k] = b;
    }
    // every finite value of the network must stay within +-2^26 so that the
    // -infinity sentinel (-2^29) plus any finite drift stays below -2^28
    int64_t total = 0;
    if (p.kind == kSpin) {
        if ((int)p.J.size() != p.m()) fail(BBTN_EINVAL, "J size");
        if (p.h2.empty()) p.h2.assign(p.n, 0);
        if ((int)p.h2.size() != p.n) fail(BBTN_EINVAL, "h2 size");
        for (auto j : p.J) {
            if (std::abs((int64_t)j) > (1 << 16)) fail(BBTN_EINVAL, "|J| > 2^16");
            total += 2 * std::abs((int64_t)j);
        }
        for (auto h : p.h2) {
            if (std::abs((int64_t)h) > (1 << 16)) fail(BBTN_EINVAL, "|h2| > 2^16");
            total += std::abs((int64_t)h);
        }
    } else {
        if (p.w.empty()) p.w.assign(p.n, 1);
        if ((int)p.w.size() != p.n) fail(BBTN_EINVAL, "w size");
        for (auto x : p.w) {
            if (x < 1 || x > (1 << 16)) fail(BBTN_EINVAL, "weight outside 1..2^16");
            total += x;
        }
    }
    if (total > (1ll << 26)) fail(BBTN_EINVAL, "sum of |entries| exceeds 2^26");
    p.build_adjacency();
}

Problem read_problem_file(const std::string &path) {
    std::ifstream f(path);
    if (!f) fail(BBTN_EIO, "cannot open " + path);
    Problem p;
    bool have_p = false;
    std::vector<std::pair<int, int>> fields, weights;
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream ss(line);
        std::string tag;
        if (!(ss >> tag) || tag == "c") continue;
        if (tag == "p") {
            std::string kind;
            int n, m;
            if (!(ss >> kind >> n >> m)) fail(BBTN_EIO, "bad p line");
            if (kind == "spin") p.kind = kSpin;
            else if (kind == "mwis") p.kind = kMwis;
            else fail(BBTN_EIO, "unknown problem kind " + kind);
            p.n = n;
            have_p = true;
        } else if (tag == "e") {
            int i, j, J = 0;
            if (!(ss >> i >> j)) fail(BBTN_EIO, "bad e line");
            if (p.kind == kSpin && !(ss >> J)) fail(BBTN_EIO, "missing coupling");
            p.ei.push_back(i);
            p.ej.push_back(j);
            if (p.kind == kSpin) p.J.push_back(J);
        } else if (tag == "f" || tag == "w") {
            int i, v;
            if (!(ss >> i >> v)) fail(BBTN_EIO, "bad f/w line");
            (tag == "f" ? fields : weights).push_back({i, v});
        } else {
            fail(BBTN_EIO, "unknown line tag " + tag);
        }
    }
    if (!have_p) fail(BBTN_EIO, "missing p line");
    if (p.kind == kSpin) {
        p.h2.assign(p.n, 0);
        for (auto &fv : fields) {
            if (fv.first < 0 || fv.first >= p.n) fail(BBTN_EIO, "field index");
            p.h2[fv.first] = fv.second;
        }
    } else {
        p.w.assign(p.n, 1);
        for (auto &wv : weights) {
            if (wv.first < 0 || wv.first >= p.n) fail(BBTN_EIO, "weight index");
            p.w[wv.first] = wv.second;
        }
    }
    validate(p);
    return p;
}

std::vector<TensorDef> build_network(const Problem &p) {
    const int32_t NEG = kNeg;
    std::vector<TensorDef> ts;
    std::vector<int> host_edge(p.n, -1);   // edge that absorbs vertex v's vector
    for (int k = 0; k < p.m(); k++) {
        if (host_edge[p.ei[k]] < 0) host_edge[p.ei[k]] = k;
        if (host_edge[p.ej[k]] < 0) host_edge[p.ej[k]] = k;
    }
    auto vertex_term = [&](int v, int x) -> int32_t {
        if (p.kind == kSpin) return (int32_t)(x ? p.h2[v] : -p.h2[v]);   // -2 w^v_s, s=0 <-> sigma=-1
        return x ? p.w[v] : 0;                                            // -w^v: (0, w_v)
    };
    for (int k = 0; k < p.m(); k++) {
        const int i = p.ei[k], j = p.ej[k];
        TensorDef t;
        t.labels = {i, j};
        t.val.resize(4);
        for (int si = 0; si < 2; si++)
            for (int sj = 0; sj < 2; sj++) {
                int32_t v;
                if (p.kind == kSpin) {
                    // -2 B^{ij}_{s_i s_j} with B = [[-J, J], [J, -J]]
                    v = 2 * p.J[k] * (2 * si - 1) * (2 * sj - 1);
                } else {
                    // -B with B = [[0, 0], [0, inf]]: both ends taken is infeasible
                    v = (si && sj) ? NEG : 0;
                }
                if (v != NEG) {
                    if (host_edge[i] == k) v += vertex_term(i, si);
                    if (host_edge[j] == k) v += vertex_term(j, sj);
                }
                t.val[si | (sj << 1)] = v;
            }
        ts.push_back(std::move(t));
    }
    for (int v = 0; v < p.n; v++)
        if (host_edge[v] < 0) {
            TensorDef t;
            t.labels = {v};
            t.val = {vertex_term(v, 0), vertex_term(v, 1)};
            ts.push_back(std::move(t));
        }
    return ts;
}

int64_t objective(const Problem &p, const std::vector<int8_t> &x) {
    int64_t s = 0;
    if (p.kind == kSpin) {
        for (int k = 0; k < p.m(); k++)
            s += 2ll * p.J[k] * (2 * x[p.ei[k]] - 1) * (2 * x[p.ej[k]] - 1);
        for (int v = 0; v < p.n; v++) s += (int64_t)p.h2[v] * (2 * x[v] - 1);
    } else {
        for (int k = 0; k < p.m(); k++)
            if (x[p.ei[k]] && x[p.ej[k]]) return INT64_MIN;
        for (int v = 0; v < p.n; v++) if (x[v]) s += p.w[v];
    }
    return s;
}

int64_t upper_bound(const Problem &p, const std::vector<int8_t> &fx) {
    int64_t ub = 0;
    if (p.kind == kSpin) {
        std::vector<int64_t> eff(p.n, 0);
        for (int v = 0; v < p.n; v++) {
            if (fx[v] >= 0) ub += (int64_t)p.h2[v] * (2 * fx[v] - 1);
            else eff[v] = p.h2[v];
        }
        for (int k = 0; k < p.m(); k++) {
            int i = p.ei[k], j = p.ej[k];
            if (fx[i] >= 0 && fx[j] >= 0) ub += 2ll * p.J[k] * (2 * fx[i] - 1) * (2 * fx[j] - 1);
            else if (fx[i] >= 0) eff[j] += 2ll * p.J[k] * (2 * fx[i] - 1);
            else if (fx[j] >= 0) eff[i] += 2ll * p.J[k] * (2 * fx[j] - 1);
            else ub += 2ll * std::abs((int64_t)p.J[k]);
        }
        for (int v = 0; v < p.n; v++) if (fx[v] < 0) ub += std::abs(eff[v]);
        return ub;
    }
    // MWIS: weight of the fixed set plus a clique-cover bound on the free vertices
    // that no fixed member excludes (an independent set meets each clique once).
    std::vector<char> allowed(p.n, 0), covered(p.n, 0);
    for (int v = 0; v < p.n; v++) {
        if (fx[v] == 1) {
            ub += p.w[v];
            for (auto &nb : p.adj[v]) if (fx[nb.first] == 1) return INT64_MIN;   // infeasible
        }
    }
    for (int v = 0; v < p.n; v++) {
        if (fx[v] != -1) continue;
        bool ok = true;
        for (auto &nb : p.adj[v]) if (fx[nb.first] == 1) { ok = false; break; }
        allowed[v] = ok;
    }
    std::vector<int> clique;
    for (int v = 0; v < p.n; v++) {
        if (!allowed[v] || covered[v]) continue;
        clique.assign(1, v);
        covered[v] = 1;
        int32_t best = p.w[v];
        for (auto &nb : p.adj[v]) {
            int u = nb.first;
            if (!allowed[u] || covered[u]) continue;
            bool all = true;
            for (int c : clique) {
                if (c == v) continue;
                bool adjc = false;
                for (auto &nb2 : p.adj[u]) if (nb2.first == c) { adjc = true; break; }
                if (!adjc) { all = false; break; }
            }
            if (all) {
                clique.push_back(u);
                covered[u] = 1;
                best = std::max(best, p.w[u]);
            }
        }
        ub += best;
    }
    return ub;
}

}  // namespace bbtn

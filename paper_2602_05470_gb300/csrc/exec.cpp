#include "exec.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <map>

#include "common.h"

namespace bbtn {

namespace {

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// First-fit allocator of byte ranges inside the arena (host-side simulation; all
// steps run in order on one stream, so a block can be reused by any step that is
// enqueued after the last reader of its previous contents).
struct FreeList {
    std::map<uint64_t, uint64_t> free_;   // offset -> size
    uint64_t top = 0, peak = 0;
    uint64_t alloc(uint64_t bytes) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                uint64_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                return off;
            }
        }
        // extend at the top (merge with a free block ending at top)
        uint64_t off = top;
        if (!free_.empty()) {
            auto last = std::prev(free_.end());
            if (last->first + last->second == top) {
                off = last->first;
                free_.erase(last);
            }
        }
        top = off + bytes;
        peak = std::max(peak, top);
        return off;
    }
    void release(uint64_t off, uint64_t bytes) {
        bytes = align256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
                it = pv;
            }
        }
        if (it->first + it->second == top) {
            top = it->first;
            free_.erase(it);
        }
    }
};

struct View {
    Ref ref;
    std::vector<int> bit_label;   // label at each physical bit, -1 for a fixed bit
    int unit = 0;
    uint64_t block_bytes = 0;     // arena block to release (kind 1)
    int free_rank() const {
        int k = 0;
        for (int l : bit_label) if (l >= 0) k++;
        return k;
    }
    int pos(int label) const {
        for (size_t i = 0; i < bit_label.size(); i++) if (bit_label[i] == label) return (int)i;
        return -1;
    }
};

void post_order(const CTree &t, std::vector<int> &order) {
    order.clear();
    std::vector<std::pair<int, int>> st{{t.root, 0}};
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
}

}  // namespace

uint64_t count_plane_offset_bytes(int r) { return align256(4ull << r); }
size_t block_bytes(int r, int np) { return count_plane_offset_bytes(r) + align256((8ull << r) * np); }

cudaEvent_t Profiler::get() {
    if (used == pool.size()) {
        cudaEvent_t e;
        BBTN_CUDA(cudaEventCreate(&e));
        pool.push_back(e);
    }
    return pool[used++];
}

void Profiler::collect() {
    for (const Rec &r : recs) {
        float t = 0;
        BBTN_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        if (dump)
            fprintf(dump, "%d,%d,%d,%d,%d,%.0f,%.0f,%.5f,%d,%d\n", r.ra, r.rb, r.rc, r.rs, r.ident, r.bytes, r.ops, t,
                    r.kind, r.n);
        bytes += r.bytes;
        ops += r.ops;
        launches++;
        if (r.kind == 0 || r.kind == 3) { stream_ms += t; stream_bytes += r.bytes; stream_launches++; }
        if (r.kind == 6) { scount_ms += t; scount_bytes += r.bytes; scount_launches++; }
        if (r.kind == 2 || r.kind == 4) { tiled_ms += t; tiled_ops += r.ops; tiled_bytes += r.bytes; tiled_launches++; }
        if (r.kind == 4) tiled16_launches++;
        if (r.kind == 5) { tcount_ms += t; tcount_ops += r.ops; tcount_bytes += r.bytes; tcount_launches++; }
        if (r.kind == 7) { chain_ms += t; chain_bytes += r.bytes; chain_launches++; }
    }
    recs.clear();
    used = 0;
}

Profiler::~Profiler() {
    if (dump) fclose(dump);
    for (auto e : pool) cudaEventDestroy(e);
}

void DeviceNetwork::set_host(const std::vector<TensorDef> &ts, int nv) {
    release();
    nvars = nv;
    offset.resize(ts.size());
    labels.resize(ts.size());
    host_vals.clear();
    value_bound = 0;
    for (size_t i = 0; i < ts.size(); i++) {
        offset[i] = host_vals.size();
        labels[i] = ts[i].labels;
        host_vals.insert(host_vals.end(), ts[i].val.begin(), ts[i].val.end());
        int64_t m = 0;
        for (int32_t v : ts[i].val)
            if (v >= kFiniteMin) m = std::max<int64_t>(m, v < 0 ? -(int64_t)v : v);
        value_bound += m;
    }
    if (host_vals.empty()) host_vals.push_back(0);
}

void DeviceNetwork::upload(cudaStream_t s) {
    if (vals) cudaFreeAsync(vals, s);   // stream-ordered: other streams keep running
    vals = nullptr;
    BBTN_CUDA(cudaMallocAsync(&vals, host_vals.size() * sizeof(int32_t), s));
    BBTN_CUDA(cudaMemcpyAsync(vals, host_vals.data(), host_vals.size() * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s));
    BBTN_CUDA(cudaStreamSynchronize(s));
}

void DeviceNetwork::release(cudaStream_t s) {
    if (vals) cudaFreeAsync(vals, s);
    vals = nullptr;
}

void Arena::reserve(size_t bytes) {
    if (bytes <= size) return;
    if (!owned) fail(BBTN_ENOMEM, "workspace too small: need " + std::to_string(bytes) + " bytes");
    if (ptr) cudaFreeAsync(ptr, stream);   // after the stream's earlier work that used it
    ptr = nullptr;
    size = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    BBTN_CUDA(cudaMallocAsync(&ptr, want, stream));
    size = want;
}

void Arena::adopt(void *p, size_t bytes) {
    release();
    ptr = (char *)p;
    size = bytes;
    owned = false;
}

void Arena::release() {
    if (ptr && owned) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
    size = 0;
    owned = true;
}

// A step that can join a K1m chain: value-only, not fused, its B operand a network
// tensor of at most 4 physical bits, at most two summed labels, four or more outputs
// (the register-tiled and split-K kernels never take such a step).
static bool chain_link(const PStep &ps) {
    if (ps.fused || !ps.P.hasB || ps.b.kind != 0 || ps.P.np != 0) return false;
    if (ps.lab_b.size() > 4 || ps.P.rs > 2 || ps.P.rc < 2) return false;
    return true;
}

// Kernel parameters of a chain from its labels: A's label at each physical bit
// (-1 fixed), and for each step the labels of B_l at its physical bits and the
// labels of the step's result. The chain's output labels are the last step's, its
// summed labels every label a step sums. False if the chain does not fit the
// kernel (too many summed labels or steps, a B of more than 4 bits).
bool chain_params(const std::vector<int> &lab_a, const std::vector<std::vector<int>> &lab_b,
                  const std::vector<std::vector<int>> &lab_c, ChainParams &cp) {
    const int L = (int)lab_b.size();
    if (L < 1 || L > kChainMaxSteps || (int)lab_c.size() != L) return false;
    const std::vector<int> &out = lab_c[L - 1];
    const int rc = (int)out.size();
    if (rc < 2 || rc > 30) return false;
    std::vector<int> S;
    for (int k = 0; k < L; k++) {
        if (lab_b[k].size() > 4) return false;
        auto in_c = [&](int l) { return std::find(lab_c[k].begin(), lab_c[k].end(), l) != lab_c[k].end(); };
        for (const auto *labs : {k == 0 ? &lab_a : &lab_c[k - 1], &lab_b[k]})
            for (int l : *labs)
                if (l >= 0 && !in_c(l) && std::find(S.begin(), S.end(), l) == S.end()) S.push_back(l);
    }
    const int rs = (int)S.size();
    if (rs > kChainMaxSum || (L << rs) > 16) return false;   // 2^rs * L add+max per output
    memset(&cp, 0, sizeof cp);
    cp.rc = rc;
    cp.rs = rs;
    cp.L = L;
    for (int q = 0; q < 32; q++) cp.oA[q] = -1;
    for (int j = 0; j < kChainMaxSum; j++) cp.sA[j] = -1;
    auto src = [&](int l) {   // output bit index, 32 + summed index, or -1
        for (int q = 0; q < rc; q++) if (out[q] == l) return q;
        for (int j = 0; j < rs; j++) if (S[j] == l) return 32 + j;
        return -1;
    };
    for (size_t q = 0; q < lab_a.size(); q++) {
        const int l = lab_a[q];
        if (l < 0) continue;
        const int w = src(l);
        if (w < 0) return false;
        if (w < 32) cp.oA[w] = (int8_t)q;
        else cp.sA[w - 32] = (int8_t)q;
    }
    for (int k = 0; k < L; k++) {
        for (size_t q = 0; q < lab_b[k].size(); q++) {
            const int l = lab_b[k][q];
            if (l < 0) continue;
            const int w = src(l);
            if (w < 0) return false;
            const uint32_t bit = 1u << (4 * k + (int)q);
            if (w < 32) cp.wC[w] += bit;
            else cp.wS[w - 32] += bit;
        }
        cp.bsize_log2[k] = (int8_t)lab_b[k].size();
    }
    return true;
}

// The chain over steps i0..i1 of a plan (step i + 1 reads step i's result as its A);
// fills the kernel parameters on step i1.
static bool build_chain(Plan &plan, int i0, int i1) {
    const int L = i1 - i0 + 1;
    if (L < 1 || L > kChainMaxSteps) return false;
    std::vector<std::vector<int>> lb, lc;
    for (int i = i0; i <= i1; i++) {
        const PStep &ps = plan.steps[i];
        lb.push_back(ps.lab_b);
        lc.emplace_back(ps.lab_c, ps.lab_c + ps.P.rc);
    }
    ChainParams cp;
    if (!chain_params(plan.steps[i0].lab_a, lb, lc, cp)) return false;
    PStep &last = plan.steps[i1];
    for (int k = 0; k < L; k++) last.chain_b[k] = plan.steps[i0 + k].b.off + plan.steps[i0 + k].b.base;
    last.chain = cp;
    last.chain_len = L;
    last.chain_first = i0;
    for (int i = i0; i < i1; i++) plan.steps[i].chain_len = -1;
    plan.chains++;
    plan.chained_steps += L;
    return true;
}

// Greedy chains over consecutive linkable steps, each step reading its
// predecessor's result as A; a run is cut where the next step would break a
// kernel limit, and only runs of two or more steps are fused.
static void find_chains(Plan &plan) {
    const int n = (int)plan.steps.size();
    int i = 0;
    while (i < n) {
        if (!chain_link(plan.steps[i]) || plan.steps[i].a.kind != 1) {
            i++;
            continue;
        }
        int j = i;
        std::vector<std::vector<int>> lb{plan.steps[i].lab_b}, lc;
        lc.emplace_back(plan.steps[i].lab_c, plan.steps[i].lab_c + plan.steps[i].P.rc);
        while (j + 1 < n && chain_link(plan.steps[j + 1]) && plan.steps[j + 1].a_node == plan.steps[j].node) {
            // extend only while the longer chain still fits the kernel
            const PStep &nx = plan.steps[j + 1];
            lb.push_back(nx.lab_b);
            lc.emplace_back(nx.lab_c, nx.lab_c + nx.P.rc);
            ChainParams probe;
            if (!chain_params(plan.steps[i].lab_a, lb, lc, probe)) break;
            j++;
        }
        if (j > i && build_chain(plan, i, j)) {
            i = j + 1;
        } else {
            i++;
        }
    }
}

// Marks the small subtrees that run fused (every step with at most 2^S outputs and
// its intermediates fitting in shared memory), lays out their shared memory, and
// assigns arena blocks in execution order: fused results first, then the other
// steps in post-order, each block released after its last reader is enqueued.
static void finalize_plan(Plan &plan, const CTree &t, int np, bool keep_all, bool chains, FreeList &fl,
                          const std::vector<char> *keep) {
    const int nsteps = (int)plan.steps.size();
    std::vector<char> fus(t.nodes.size(), 0);
    const int S = np == 0 ? 14 : 11;
    const uint64_t budget = 200 * 1024;
    if (!keep_all && np <= 4) {
        for (int i = 0; i < nsteps; i++) {
            const PStep &ps = plan.steps[i];
            if (t.nodes[ps.node].is_leaf()) continue;
            bool ok = ps.P.rc <= S && ps.P.rs <= 12;
            for (int c : {ps.a_node, ps.b_node})
                if (c >= 0 && !t.nodes[c].is_leaf() && !fus[c]) ok = false;
            fus[ps.node] = ok;
        }
    }
    auto nint = [&](int n) {   // internal nodes of a fused subtree
        int c = 0;
        std::vector<int> st{n};
        while (!st.empty()) {
            int x = st.back();
            st.pop_back();
            if (t.nodes[x].is_leaf()) continue;
            c++;
            st.push_back(t.nodes[x].l);
            st.push_back(t.nodes[x].r);
        }
        return c;
    };
    std::vector<int> roots;
    std::vector<uint32_t> soff(t.nodes.size(), 0);
    for (bool changed = true; changed;) {
        changed = false;
        roots.clear();
        for (int i = 0; i < nsteps; i++) {
            const int n = plan.steps[i].node;
            const int par = t.nodes[n].parent;
            if (fus[n] && (par < 0 || !fus[par])) roots.push_back(n);
        }
        plan.fused_smem = 0;
        for (int r : roots) {
            const int last = plan.node_step[r], first = last - nint(r) + 1;
            FreeList fsm;
            for (int i = first; i <= last; i++) {
                const PStep &ps = plan.steps[i];
                if (ps.node != r) soff[ps.node] = (uint32_t)fsm.alloc(smem_tensor_bytes(ps.P.rc, np));
                for (int c : {ps.a_node, ps.b_node})
                    if (c >= 0 && !t.nodes[c].is_leaf())
                        fsm.release(soff[c], smem_tensor_bytes(plan.steps[plan.node_step[c]].P.rc, np));
            }
            if (fsm.peak > budget) {
                fus[r] = 0;
                changed = true;
            }
            plan.fused_smem = std::max<size_t>(plan.fused_smem, fsm.peak);
        }
    }
    for (int i = 0; i < nsteps; i++)
        if (fus[plan.steps[i].node]) plan.steps[i].fused = true;
    if (chains && np == 0 && !keep_all) {
        find_chains(plan);
        // the fused chain moves A once and C once instead of every intermediate
        for (int i = 0; i < nsteps; i++) {
            PStep &ps = plan.steps[i];
            if (ps.chain_len == 0) continue;
            plan.bytes -= ps.bytes;
            if (ps.chain_len > 0) {
                const PStep &f = plan.steps[ps.chain_first];
                int ra = 0;
                for (int l : f.lab_a) ra += l >= 0;
                ps.bytes = std::ldexp(4.0, ra) + std::ldexp(4.0, ps.P.rc);
                plan.bytes += ps.bytes;
            } else {
                ps.bytes = 0;
            }
        }
    }
    // arena: fused results are alive from the fused launch on
    for (int r : roots)
        if (r != t.root) {
            PStep &ps = plan.steps[plan.node_step[r]];
            ps.c.off = fl.alloc(ps.c_block);
        }
    for (int i = 0; i < nsteps; i++) {
        PStep &ps = plan.steps[i];
        if (ps.fused) continue;
        if (ps.chain_len < 0) continue;   // inside a chain: nothing materialised, A stays alive
        if (ps.c.kind == 1) ps.c.off = fl.alloc(ps.c_block);
        if (ps.chain_len > 0) {
            // the chain reads its first step's A (released only now, after C is placed,
            // so that C never takes A's block) and network tensors
            const PStep &f = plan.steps[ps.chain_first];
            ps.chain_a = f.a;
            const int c = f.a_node;
            if (c >= 0 && !t.nodes[c].is_leaf()) {
                const PStep &cs = plan.steps[plan.node_step[c]];
                ps.chain_a = cs.c;
                fl.release(cs.c.off, cs.c_block);
            }
            continue;
        }
        for (int side = 0; side < 2; side++) {
            const int c = side ? ps.b_node : ps.a_node;
            if (c < 0 || t.nodes[c].is_leaf() || (side == 1 && !ps.P.hasB)) continue;
            const PStep &cs = plan.steps[plan.node_step[c]];
            (side ? ps.b : ps.a) = cs.c;
            if (!keep_all || (keep && !(*keep)[c])) fl.release(cs.c.off, cs.c_block);
        }
    }
    plan.arena_bytes = fl.peak;
    // one shared scratch region for the split-K steps (they run one after another)
    for (int i = 0; i < nsteps; i++) {
        const PStep &ps = plan.steps[i];
        if (!ps.fused && splitk_eligible(ps.P))
            plan.splitk_bytes = std::max<uint64_t>(plan.splitk_bytes, splitk_scratch_bytes(ps.P.rc, np));
    }
    if (plan.splitk_bytes) {
        plan.splitk_off = align256(plan.arena_bytes);
        plan.arena_bytes = plan.splitk_off + plan.splitk_bytes;
    }
    // the fused program
    for (int r : roots) {
        const int last = plan.node_step[r], first = last - nint(r) + 1;
        FSub sub;
        sub.first = (int)plan.fsteps.size();
        sub.count = last - first + 1;
        sub.leaf = 0;
        for (int i = first; i <= last; i++) {
            const PStep &ps = plan.steps[i];
            FStep f;
            memset(&f, 0, sizeof f);
            f.rc = (int8_t)ps.P.rc;
            f.rs = (int8_t)ps.P.rs;
            f.hasB = (int8_t)ps.P.hasB;
            for (int q = 0; q < kFusedMaxBits; q++) {
                f.oA[q] = ps.P.oA[q];
                f.oB[q] = ps.P.oB[q];
                f.sA[q] = ps.P.sA[q];
                f.sB[q] = ps.P.sB[q];
            }
            for (int side = 0; side < 2; side++) {
                const int c = side ? ps.b_node : ps.a_node;
                if (side == 1 && !ps.P.hasB) continue;
                const Ref &rf = side ? ps.b : ps.a;
                int8_t kind, rank = 0;
                uint32_t off;
                if (c < 0 || t.nodes[c].is_leaf()) {
                    kind = 0;
                    off = (uint32_t)(rf.off + rf.base);
                } else {
                    kind = 1;
                    off = soff[c];
                    rank = (int8_t)plan.steps[plan.node_step[c]].P.rc;
                }
                if (side) { f.b_kind = kind; f.b_off = off; f.b_rank = rank; }
                else { f.a_kind = kind; f.a_off = off; f.a_rank = rank; }
            }
            if (ps.node != r) {
                f.c_kind = 1;
                f.c_off = soff[ps.node];
            } else if (r == t.root) {
                f.c_kind = 3;
            } else {
                f.c_kind = 2;
                f.c_goff = ps.c.off;
            }
            plan.fsteps.push_back(f);
            plan.fused_steps++;
        }
        plan.fsubs.push_back(sub);
    }
}

static Plan make_plan_impl(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx, int np,
                           const uint32_t *cprime, bool keep_all, bool chains, FreeList &fl,
                           const std::vector<char> *keep);

Plan make_plan(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx, int np,
               const uint32_t *cprime, bool keep_all, bool chains) {
    FreeList fl;
    return make_plan_impl(t, net, fx, np, cprime, keep_all, chains, fl, nullptr);
}

static Plan make_plan_impl(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx, int np,
                           const uint32_t *cprime, bool keep_all, bool chains, FreeList &fl,
                           const std::vector<char> *keep) {
    Plan plan;
    plan.np = np;
    plan.node_step.assign(t.nodes.size(), -1);
    plan.node_layout.assign(t.nodes.size(), {});
    std::vector<View> view(t.nodes.size());
    std::vector<int> order;
    post_order(t, order);
    const uint64_t elem = 4 + 8ull * np;

    // Layout policy: each result orders its labels by the step at which they are
    // next active (summed, or shared with the partner operand) -- latest first, so
    // the low bits of a tensor are labels that its consumer passes through. The
    // consumer's reads of its big operand then coalesce along those low bits.
    std::vector<int> pos(t.nodes.size(), 0);
    for (size_t i = 0; i < order.size(); i++) pos[order[i]] = (int)i;
    std::vector<std::vector<int>> key(t.nodes.size());
    {
        std::vector<int> stack{t.root};
        key[t.root].assign(t.nodes[t.root].lab.size(), (int)order.size());
        while (!stack.empty()) {
            const int q = stack.back();
            stack.pop_back();
            const CNode &nq = t.nodes[q];
            if (nq.is_leaf()) continue;
            for (int side = 0; side < 2; side++) {
                const int a = side ? nq.r : nq.l, b = side ? nq.l : nq.r;
                const auto &la = t.nodes[a].lab, &lb = t.nodes[b].lab;
                key[a].resize(la.size());
                for (size_t i = 0; i < la.size(); i++) {
                    const int l = la[i];
                    auto it = std::lower_bound(nq.lab.begin(), nq.lab.end(), l);
                    const bool in_q = it != nq.lab.end() && *it == l;
                    if (!in_q || std::binary_search(lb.begin(), lb.end(), l)) key[a][i] = pos[q];
                    else key[a][i] = key[q][it - nq.lab.begin()];
                }
                stack.push_back(a);
            }
        }
    }
    auto key_of = [&](int node, int l) {
        const auto &lab = t.nodes[node].lab;
        auto it = std::lower_bound(lab.begin(), lab.end(), l);
        return key[node][it - lab.begin()];
    };

    auto leaf_view = [&](int id) {
        const CNode &nd = t.nodes[id];
        View v;
        v.ref.kind = 0;
        v.ref.off = net.offset[nd.leaf];
        v.unit = 1;
        const auto &labs = net.labels[nd.leaf];
        for (size_t i = 0; i < labs.size(); i++) {
            int l = labs[i];
            if (fx[l] >= 0) {
                v.ref.base += (uint64_t)fx[l] << i;
                v.bit_label.push_back(-1);
            } else {
                v.bit_label.push_back(l);
            }
        }
        return v;
    };

    auto emit = [&](int id, const View *X, const View *Y, bool is_root) {
        // A: the operand with more free elements (reads coalesce along its low bits)
        const View *A = X, *B = Y;
        const CNode &nd0 = t.nodes[id];
        int a_node = nd0.is_leaf() ? id : nd0.l, b_node = nd0.is_leaf() ? -1 : nd0.r;
        if (B && B->free_rank() > A->free_rank()) {
            std::swap(A, B);
            std::swap(a_node, b_node);
        }
        const CNode &nd = t.nodes[id];
        auto kept = [&](int l) { return std::binary_search(nd.lab.begin(), nd.lab.end(), l); };
        std::vector<int> out, sum;
        for (int l : A->bit_label) if (l >= 0) (kept(l) ? out : sum).push_back(l);
        if (B)
            for (int l : B->bit_label)
                if (l >= 0 && A->pos(l) < 0) (kept(l) ? out : sum).push_back(l);
        if (!is_root)
            std::stable_sort(out.begin(), out.end(),
                             [&](int x, int y) { return key_of(id, x) > key_of(id, y); });
        if (out.size() > 30) fail(BBTN_ENOMEM, "intermediate rank above 30");
        if (sum.size() > 40) fail(BBTN_ENOMEM, "more than 40 summed labels in one step");
        PStep st;
        st.node = id;
        st.a_node = a_node;
        st.b_node = b_node;
        ContractParams &P = st.P;
        P.rc = (int)out.size();
        P.rs = (int)sum.size();
        P.hasB = B != nullptr;
        P.np = np;
        // every finite entry of an intermediate is a sum of one entry per network
        // tensor, so |value| <= value_bound: 16-bit lanes are exact below 2^12
        P.v16 = np == 0 && net.value_bound < (1 << 12);
        for (int t2 = 0; t2 < np; t2++) P.cprime[t2] = cprime[t2];
        for (int i = 0; i < 32; i++) P.oA[i] = P.oB[i] = P.sA[i] = P.sB[i] = -1;
        for (int i = 0; i < P.rc; i++) {
            P.oA[i] = (int8_t)A->pos(out[i]);
            P.oB[i] = B ? (int8_t)B->pos(out[i]) : -1;
            st.lab_c[i] = out[i];
        }
        if (P.rs > 32) fail(BBTN_ENOMEM, "more than 32 summed labels in one step");
        for (int j = 0; j < P.rs; j++) {
            P.sA[j] = (int8_t)A->pos(sum[j]);
            P.sB[j] = B ? (int8_t)B->pos(sum[j]) : -1;
        }
        st.a = A->ref;
        st.lab_a = A->bit_label;
        P.A.unit_counts = A->unit;
        if (B) {
            st.b = B->ref;
            st.lab_b = B->bit_label;
            P.B.unit_counts = B->unit;
        }
        View C;
        C.bit_label = out;
        if (is_root) {
            C.ref.kind = 2;
        } else {
            C.ref.kind = 1;
            C.block_bytes = block_bytes(P.rc, np);
            C.ref.off = 0;                     // assigned by the allocation pass below
            C.ref.plane = 1ull << P.rc;
            C.ref.rank = P.rc;
        }
        st.c = C.ref;
        st.ops = std::ldexp(1.0, P.rc + P.rs);
        st.bytes = std::ldexp((double)(A->unit ? 4 : elem), A->free_rank()) +
                   (B ? std::ldexp((double)(B->unit ? 4 : elem), B->free_rank()) : 0.0) +
                   std::ldexp((double)elem, P.rc);
        plan.ops += st.ops;
        plan.bytes += st.bytes;
        plan.max_rank = std::max(plan.max_rank, P.rc);
        st.c_block = C.block_bytes;
        plan.node_step[id] = (int)plan.steps.size();
        plan.node_layout[id] = out;
        plan.steps.push_back(st);
        return C;
    };

    for (int id : order) {
        const CNode &nd = t.nodes[id];
        if (nd.is_leaf()) {
            view[id] = leaf_view(id);
            if (id == t.root) emit(id, &view[id], nullptr, true);   // single-tensor network
            continue;
        }
        view[id] = emit(id, &view[nd.l], &view[nd.r], id == t.root);
        if (!keep_all) {
            view[nd.l].bit_label.clear();
            view[nd.r].bit_label.clear();
        }
    }
    finalize_plan(plan, t, np, keep_all, chains, fl, keep);
    return plan;
}

static void fill_operand(Operand &o, const Ref &r, const DeviceNetwork &net, char *arena) {
    if (r.kind == 0) {
        o.val = net.vals + r.off;
        o.cnt = nullptr;
        o.plane = 0;
        o.base = r.base;
    } else {
        o.val = (const int32_t *)(arena + r.off);
        o.cnt = (const uint64_t *)(arena + r.off + count_plane_offset_bytes(r.rank));
        o.plane = r.plane;
        o.base = 0;
    }
}

void DeviceBuf::reserve(size_t bytes) {
    if (bytes <= size) return;
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
    size = 0;
    const size_t want = std::max(bytes * 2, (size_t)1 << 20);
    BBTN_CUDA(cudaMallocAsync(&ptr, want, stream));
    size = want;
}

DeviceBuf::~DeviceBuf() {
    if (ptr) cudaFreeAsync(ptr, stream);
}

namespace {

struct LaunchTimer {
    Profiler *pr;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer(Profiler *p, cudaStream_t st) : pr(p), s(st) {
        if (pr) {
            a = pr->get();
            b = pr->get();
            BBTN_CUDA(cudaEventRecord(a, s));
        }
    }
    void done(double bytes, double ops, const ContractParams *P, int kind, int n) {
        if (!pr) return;
        if (kind == 2 && P) kind = P->np > 0 ? 5 : (tiled_uses_v16(*P) ? 4 : 2);
        if ((kind == 0 || kind == 3) && P && P->np > 0) kind = 6;
        BBTN_CUDA(cudaEventRecord(b, s));
        int ra = 0, rb = 0, ident = 0, rc = 0, rs = 0;
        if (P) {
            for (int i = 0; i < P->rc; i++) { if (P->oA[i] >= 0) ra++; if (P->oB[i] >= 0) rb++; }
            for (int j = 0; j < P->rs; j++) { if (P->sA[j] >= 0) ra++; if (P->sB[j] >= 0) rb++; }
            while (ident < P->rc && P->oA[ident] == ident && P->oB[ident] < 0) ident++;
            rc = P->rc;
            rs = P->rs;
        }
        pr->recs.push_back({a, b, bytes, ops, ra, rb, rc, rs, ident, kind, n});
    }
};

// Shape class of a tiled step: the group sizes (batch, m, n, k) and the role
// (free in one operand, batch, summed, absent) of each operand's two lowest bits --
// what decides how its loads coalesce. Leaves of one tree give the same few classes.
uint64_t step_signature(const ContractParams &P) {
    int nb = 0, nm = 0, nn = 0;
    for (int i = 0; i < P.rc; i++) {
        if (P.oA[i] >= 0 && P.oB[i] >= 0) nb++;
        else if (P.oA[i] >= 0) nm++;
        else nn++;
    }
    auto role = [&](const int8_t *o, const int8_t *other, const int8_t *sm, int q) {
        for (int i = 0; i < P.rc; i++)
            if (o[i] == q) return other[i] >= 0 ? 2 : 1;   // batch / free
        for (int j = 0; j < P.rs; j++)
            if (sm[j] == q) return 3;                       // summed
        return 0;
    };
    uint64_t h = (uint64_t)P.np | (uint64_t)P.v16 << 4 | (uint64_t)nb << 8 | (uint64_t)nm << 16 |
                 (uint64_t)nn << 24 | (uint64_t)P.rs << 32;
    h |= (uint64_t)role(P.oA, P.oB, P.sA, 0) << 40 | (uint64_t)role(P.oA, P.oB, P.sA, 1) << 42;
    h |= (uint64_t)role(P.oB, P.oA, P.sB, 0) << 44 | (uint64_t)role(P.oB, P.oA, P.sB, 1) << 46;
    return h;
}

}  // namespace

int TileTuner::pick(uint64_t key, const std::function<cudaError_t(int)> &launch, cudaStream_t s) {
    auto it = best.find(key);
    if (it != best.end()) return it->second;
    if (!ev[0]) {
        BBTN_CUDA(cudaEventCreate(&ev[0]));
        BBTN_CUDA(cudaEventCreate(&ev[1]));
    }
    // two rounds in opposite orders, each candidate's faster time counts: the first
    // launch finds the operands outside L2, so a single round favours the later ones
    float t[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int round = 0; round < 2; round++)
        for (int i = 0; i < 4; i++) {
            const int l = round ? 3 - i : i;
            BBTN_CUDA(cudaEventRecord(ev[0], s));
            cudaError_t e = launch(l);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("tiled (tuning): ") + cudaGetErrorString(e));
            BBTN_CUDA(cudaEventRecord(ev[1], s));
            BBTN_CUDA(cudaEventSynchronize(ev[1]));
            float ms = 0;
            BBTN_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            t[l] = std::min(t[l], ms);
        }
    int choice = 0;
    for (int l = 1; l < 4; l++)
        if (t[l] < t[choice]) choice = l;
    best[key] = choice;
    tuned++;
    return choice;
}

TileTuner::~TileTuner() {
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
}

void run_plans(const std::vector<const Plan *> &plans, const DeviceNetwork &net, char *arena, uint64_t stride,
               int32_t *out_val, uint64_t *out_cnt, uint64_t out_plane, cudaStream_t s, RunStats *st,
               DeviceBuf *prog) {
    const int nl = (int)plans.size();
    if (nl == 0) return;
    if (nl > kBatchMax) fail(BBTN_EINVAL, "run_plans: too many leaves in one batch");
    const int np = plans[0]->np;
    Profiler *pr = st ? st->prof : nullptr;
    // ---- all small subtrees of every leaf in one launch (K5)
    {
        std::vector<FStep> fsteps;
        std::vector<FSub> fsubs;
        size_t smem = 0;
        for (int i = 0; i < nl; i++) {
            const Plan &pl = *plans[i];
            const int base = (int)fsteps.size();
            fsteps.insert(fsteps.end(), pl.fsteps.begin(), pl.fsteps.end());
            for (FSub sub : pl.fsubs) {
                sub.first += base;
                sub.leaf = i;
                fsubs.push_back(sub);
            }
            smem = std::max(smem, pl.fused_smem);
        }
        if (!fsubs.empty()) {
            const size_t bs = fsteps.size() * sizeof(FStep);
            const size_t bsub = fsubs.size() * sizeof(FSub);
            const size_t off_sub = (bs + 255) & ~(size_t)255;
            prog->reserve(off_sub + bsub);
            BBTN_CUDA(cudaMemcpyAsync(prog->ptr, fsteps.data(), bs, cudaMemcpyHostToDevice, s));
            BBTN_CUDA(cudaMemcpyAsync((char *)prog->ptr + off_sub, fsubs.data(), bsub, cudaMemcpyHostToDevice, s));
            FusedParams fp{};
            fp.steps = (const FStep *)prog->ptr;
            fp.subs = (const FSub *)((char *)prog->ptr + off_sub);
            fp.nsubs = (int)fsubs.size();
            fp.net = net.vals;
            fp.arena = arena;
            fp.arena_stride = stride;
            fp.out_val = out_val;
            fp.out_cnt = out_cnt;
            fp.out_plane = out_plane;
            fp.np = np;
            for (int t2 = 0; t2 < np; t2++) fp.cprime[t2] = plans[0]->steps.empty() ? 0 : plans[0]->steps[0].P.cprime[t2];
            LaunchTimer lt(pr, s);
            cudaError_t e = launch_fused(fp, smem, s);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("fused kernel: ") + cudaGetErrorString(e));
            lt.done(0.0, 0.0, nullptr, 1, nl);
            if (st) st->launches++;
        }
    }
    // ---- the remaining steps in post-order; the step of one tree node for every
    // leaf of the batch goes out in one launch per kernel
    const size_t nsteps = plans[0]->steps.size();
    for (int i = 1; i < nl; i++)
        if (plans[i]->steps.size() != nsteps) fail(BBTN_ESTATE, "run_plans: plans of different trees");
    std::vector<ContractParams> tiled, strm;
    std::vector<ChainParams> chain[kChainMaxSteps + 1];
    double c_bytes[kChainMaxSteps + 1], c_ops[kChainMaxSteps + 1];
    std::vector<double> tb, tops, sb, sops;
    for (size_t k = 0; k < nsteps; k++) {
        tiled.clear();
        strm.clear();
        for (int l = 0; l <= kChainMaxSteps; l++) {
            chain[l].clear();
            c_bytes[l] = c_ops[l] = 0;
        }
        double t_bytes = 0, t_ops = 0, s_bytes = 0, s_ops = 0;
        for (int i = 0; i < nl; i++) {
            const Plan &pl = *plans[i];
            const PStep &ps = pl.steps[k];
            if (ps.node != plans[0]->steps[k].node) fail(BBTN_ESTATE, "run_plans: plans of different trees");
            if (ps.fused || ps.chain_len < 0) continue;
            char *ar = arena + (uint64_t)i * stride;
            if (ps.chain_len > 0) {
                ChainParams cp = ps.chain;
                Operand a;
                fill_operand(a, ps.chain_a, net, ar);
                cp.a = a.val + a.base;
                cp.vc = ps.c.kind == 2 ? out_val + i : (int32_t *)(ar + ps.c.off);
                for (int l = 0; l < cp.L; l++) cp.b[l] = net.vals + ps.chain_b[l];
                chain[cp.L].push_back(cp);
                c_bytes[cp.L] += ps.bytes;
                for (int j = ps.chain_first; j <= (int)k; j++) c_ops[cp.L] += pl.steps[j].ops;
                if (st) {
                    st->chains++;
                    st->chained_steps += cp.L;
                }
                continue;
            }
            ContractParams P = ps.P;
            fill_operand(P.A, ps.a, net, ar);
            P.A.unit_counts = ps.a.kind == 0;
            if (P.hasB) {
                fill_operand(P.B, ps.b, net, ar);
                P.B.unit_counts = ps.b.kind == 0;
            }
            if (ps.c.kind == 2) {
                P.vc = out_val + i;
                P.cc = out_cnt ? out_cnt + i : nullptr;
                P.planeC = out_plane;
            } else {
                P.vc = (int32_t *)(ar + ps.c.off);
                P.cc = (uint64_t *)(ar + ps.c.off + count_plane_offset_bytes(P.rc));
                P.planeC = 1ull << P.rc;
            }
            void *scratch = pl.splitk_bytes ? ar + pl.splitk_off : nullptr;
            if (!(scratch && splitk_eligible(P))) {
                if (tiled_eligible(P)) {
                    tiled.push_back(P);
                    t_bytes += ps.bytes;
                    t_ops += ps.ops;
                    continue;
                }
                if (stream4_eligible(P)) {
                    strm.push_back(P);
                    s_bytes += ps.bytes;
                    s_ops += ps.ops;
                    continue;
                }
            }
            LaunchTimer lt(pr, s);
            int kind = 0;
            cudaError_t e = launch_contract(P, s, &kind, scratch, pl.splitk_bytes);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("contract kernel: ") + cudaGetErrorString(e));
            lt.done(ps.bytes, ps.ops, &P, kind, 1);
            if (st) st->launches++;
        }
        if (!tiled.empty()) {
            int lanes = -1;
            if (st && st->tuner)   // timed on the first leaf's step alone
                lanes = st->tuner->pick(step_signature(tiled[0]),
                                        [&](int l) { return launch_contract_tiled_batch(tiled.data(), 1, s, l); }, s);
            LaunchTimer lt(pr, s);
            cudaError_t e = launch_contract_tiled_batch(tiled.data(), (int)tiled.size(), s, lanes);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("tiled batch: ") + cudaGetErrorString(e));
            lt.done(t_bytes, t_ops, &tiled[0], 2, (int)tiled.size());
            if (st) st->launches++;
        }
        if (!strm.empty()) {
            LaunchTimer lt(pr, s);
            cudaError_t e = launch_contract_stream4_batch(strm.data(), (int)strm.size(), s);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("stream batch: ") + cudaGetErrorString(e));
            lt.done(s_bytes, s_ops, &strm[0], 0, (int)strm.size());
            if (st) st->launches++;
        }
        for (int l = 1; l <= kChainMaxSteps; l++) {
            if (chain[l].empty()) continue;
            LaunchTimer lt(pr, s);
            cudaError_t e = launch_chain_batch(chain[l].data(), (int)chain[l].size(), s);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("chain batch: ") + cudaGetErrorString(e));
            lt.done(c_bytes[l], c_ops[l], nullptr, 7, (int)chain[l].size());
            if (st) st->launches++;
        }
    }
    if (st)
        for (const Plan *pl : plans) {
            st->ops += pl->ops;
            st->bytes += pl->bytes;
        }
}

void run_plan(const Plan &plan, const DeviceNetwork &net, char *arena, int32_t *out_val,
              uint64_t *out_cnt, uint64_t out_plane, cudaStream_t s, RunStats *st, DeviceBuf *prog) {
    run_plans({&plan}, net, arena, 0, out_val, out_cnt, out_plane, s, st, prog);
}

namespace {

// The walk of a backward plan for a given checkpoint set, simulated on the host
// allocator that the forward left behind.
void plan_walk(BackwardPlan &bp, const CTree &t, const std::vector<char> &keep, FreeList &fl) {
    const Plan &pl = bp.fwd;
    const int nn = (int)t.nodes.size();
    std::vector<char> avail(nn, 0);
    std::vector<Ref> cur(nn);
    bp.actions.clear();
    bp.recomputed = 0;
    auto internal = [&](int c) { return c >= 0 && !t.nodes[c].is_leaf(); };
    for (int n = 0; n < nn; n++)
        if (internal(n) && keep[n] && pl.node_step[n] >= 0) {
            avail[n] = 1;
            cur[n] = pl.steps[pl.node_step[n]].c;
        }
    auto operand = [&](const PStep &ps, int side) {
        const int c = side ? ps.b_node : ps.a_node;
        return internal(c) && c != t.root ? cur[c] : (side ? ps.b : ps.a);
    };
    // recompute the segment below c: every unavailable internal node reachable
    // from c without passing an available one, in post-order
    std::function<void(int)> recompute = [&](int c) {
        if (!internal(c) || avail[c]) return;
        const PStep &ps = pl.steps[pl.node_step[c]];
        recompute(ps.a_node);
        if (ps.P.hasB) recompute(ps.b_node);
        BwdAction ac;
        ac.kind = 0;
        ac.node = c;
        ac.a = operand(ps, 0);
        if (ps.P.hasB) ac.b = operand(ps, 1);
        ac.c = ps.c;
        ac.c.off = fl.alloc(ps.c_block);
        cur[c] = ac.c;
        avail[c] = 1;
        bp.actions.push_back(ac);
        bp.recomputed++;
    };
    std::vector<int> stack{t.root};
    while (!stack.empty()) {
        const int n = stack.back();
        stack.pop_back();
        const PStep &ps = pl.steps[pl.node_step[n]];
        if (internal(ps.a_node) && ps.a_node != n) recompute(ps.a_node);
        if (ps.P.hasB && internal(ps.b_node)) recompute(ps.b_node);
        BwdAction ac;
        ac.kind = 1;
        ac.node = n;
        ac.a = operand(ps, 0);
        if (ps.P.hasB) ac.b = operand(ps, 1);
        ac.c = n == t.root ? ps.c : cur[n];
        bp.actions.push_back(ac);
        if (n != t.root) fl.release(cur[n].off, ps.c_block);   // its own backward was its last reader
        if (ps.P.hasB && internal(ps.b_node)) stack.push_back(ps.b_node);
        if (internal(ps.a_node) && ps.a_node != n) stack.push_back(ps.a_node);
    }
}

}  // namespace

BackwardPlan make_backward_plan(const CTree &t, const DeviceNetwork &net, const std::vector<int8_t> &fx,
                                uint64_t budget) {
    const int nn = (int)t.nodes.size();
    std::vector<char> keep(nn, 1);
    BackwardPlan best;
    bool have = false;
    // sizes of the intermediates (values only), from the plan that keeps them all
    Plan all = make_plan(t, net, fx, 0, nullptr, true, false);
    std::vector<double> size(nn, 0.0);
    double largest = 0;
    for (const PStep &ps : all.steps)
        if (ps.c.kind == 1) {
            size[ps.node] = (double)ps.c_block;
            largest = std::max(largest, size[ps.node]);
        }
    // checkpoints for a segment budget S: post-order, a node's segment is itself plus
    // its children's unkept segments; while it exceeds S the child with the largest
    // segment becomes a checkpoint. S = infinity keeps everything (no recompute).
    std::vector<int> order;
    post_order(t, order);
    double total = 0;
    for (double x : size) total += x;
    // segment sizes from the whole tree (keep everything) down to the largest tensor:
    // the first plan within the budget recomputes least; else the smallest peak
    for (double S = INFINITY;; S = std::isinf(S) ? total / 2 : S / 2) {
        std::vector<double> acc(nn, 0.0);
        std::fill(keep.begin(), keep.end(), 0);
        for (int n : order) {
            if (t.nodes[n].is_leaf()) continue;
            const int l = t.nodes[n].l, r = t.nodes[n].r;
            double a = size[n] + acc[l] + acc[r];
            while (a > S) {
                const int c = acc[l] >= acc[r] ? l : r;
                if (acc[c] <= 0) break;
                keep[c] = 1;
                a -= acc[c];
                acc[c] = 0;
            }
            acc[n] = a;
        }
        if (std::isinf(S))
            for (int n = 0; n < nn; n++) keep[n] = !t.nodes[n].is_leaf();
        BackwardPlan bp;
        FreeList fl;
        bp.fwd = make_plan_impl(t, net, fx, 0, nullptr, true, false, fl, &keep);
        plan_walk(bp, t, keep, fl);
        bp.peak_bytes = (double)fl.peak;
        bp.keep_all_bytes = (double)all.arena_bytes;
        bp.kept = 0;
        for (int n = 0; n < nn; n++) bp.kept += keep[n] && !t.nodes[n].is_leaf() && n != t.root;
        const bool fits = bp.peak_bytes <= (double)budget;
        if (!have || fits || bp.peak_bytes < best.peak_bytes) {
            best = std::move(bp);
            have = true;
        }
        if (fits || S < largest) break;
    }
    // the selection array and the split-K scratch after the tensors
    uint64_t top = align256((uint64_t)best.peak_bytes);
    best.sel_off = top;
    top = align256(top + 8ull * (nn + 1));
    for (const PStep &ps : best.fwd.steps)
        if (splitk_eligible(ps.P)) best.scratch_bytes = std::max<uint64_t>(best.scratch_bytes, splitk_scratch_bytes(ps.P.rc, 0));
    best.scratch_off = top;
    best.arena_bytes = top + best.scratch_bytes;
    // the forward's own split-K scratch sits at its plan's offset: keep it inside the arena
    best.arena_bytes = std::max<size_t>(best.arena_bytes, best.fwd.arena_bytes);
    return best;
}

void run_backward(const BackwardPlan &bp, const CTree &t, const DeviceNetwork &net, char *arena,
                  int32_t *root_val, const std::vector<int8_t> &fx, std::vector<int8_t> &x, cudaStream_t s,
                  RunStats *st, DeviceBuf *prog) {
    run_plan(bp.fwd, net, arena, root_val, nullptr, 0, s, st, prog);
    const int nn = (int)t.nodes.size();
    int64_t *dsel = (int64_t *)(arena + bp.sel_off);
    BBTN_CUDA(cudaMemsetAsync(dsel, 0xff, 8ull * (nn + 1), s));          // -1: not selected
    BBTN_CUDA(cudaMemsetAsync(dsel + t.root, 0, 8, s));                   // the root scalar
    void *scratch = bp.scratch_bytes ? arena + bp.scratch_off : nullptr;
    for (const BwdAction &ac : bp.actions) {
        const PStep &ps = bp.fwd.steps[bp.fwd.node_step[ac.node]];
        ContractParams P = ps.P;
        fill_operand(P.A, ac.a, net, arena);
        P.A.unit_counts = ac.a.kind == 0;
        if (P.hasB) {
            fill_operand(P.B, ac.b, net, arena);
            P.B.unit_counts = ac.b.kind == 0;
        }
        if (ac.kind == 0) {
            P.vc = (int32_t *)(arena + ac.c.off);
            P.cc = nullptr;
            P.planeC = 1ull << P.rc;
            int kind = 0;
            cudaError_t e = launch_contract(P, s, &kind, scratch, bp.scratch_bytes);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("backward recompute: ") + cudaGetErrorString(e));
        } else {
            BackwardParams B;
            B.va = P.A.val;
            B.vb = P.hasB ? P.B.val : nullptr;
            B.baseA = P.A.base;
            B.baseB = P.hasB ? P.B.base : 0;
            B.vc = ac.c.kind == 2 ? root_val : (const int32_t *)(arena + ac.c.off);
            B.rc = P.rc;
            B.rs = P.rs;
            B.hasB = P.hasB;
            memcpy(B.oA, P.oA, 32);
            memcpy(B.oB, P.oB, 32);
            memcpy(B.sA, P.sA, 32);
            memcpy(B.sB, P.sB, 32);
            int64_t *sb = P.hasB && ps.b_node >= 0 ? dsel + ps.b_node : dsel + nn;
            cudaError_t e = launch_backward(B, 1, dsel + ac.node, dsel + ps.a_node, sb, s);
            if (e != cudaSuccess) fail(BBTN_ECUDA, std::string("backward kernel: ") + cudaGetErrorString(e));
        }
        if (st) st->launches++;
    }
    std::vector<int64_t> sel(nn + 1);
    BBTN_CUDA(cudaMemcpyAsync(sel.data(), dsel, 8ull * (nn + 1), cudaMemcpyDeviceToHost, s));
    BBTN_CUDA(cudaStreamSynchronize(s));
    x = fx;
    for (int n = 0; n < nn; n++) {
        if (!t.nodes[n].is_leaf()) continue;
        const int64_t idx = sel[n];
        if (idx < 0) fail(BBTN_ESTATE, "backward: no maximising assignment (infeasible)");
        const auto &labs = net.labels[t.nodes[n].leaf];
        for (size_t i = 0; i < labs.size(); i++)
            if (fx[labs[i]] < 0) x[labs[i]] = (int8_t)((idx >> i) & 1);
    }
}

}  // namespace bbtn

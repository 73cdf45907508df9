#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.h"
#include "gnn.h"

namespace bbtn {

namespace {

int din_of(int l) { return l == 0 ? kGnnFeat : kGnnHidden; }

// offsets of W_l, U_l, b_l and of the head
struct Layout {
    int W[kGnnLayers], U[kGnnLayers], b[kGnnLayers], w, c, total;
    Layout() {
        int off = 0;
        for (int l = 0; l < kGnnLayers; l++) {
            const int d = din_of(l);
            W[l] = off;
            U[l] = off + d * kGnnHidden;
            b[l] = off + 2 * d * kGnnHidden;
            off += 2 * d * kGnnHidden + kGnnHidden;
        }
        w = off;
        c = off + kGnnHidden;
        total = c + 1;
    }
};
const Layout &layout() {
    static Layout L;
    return L;
}

#define GNN_CHECK(x)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) fail(BBTN_ECUDA, std::string("gnn: ") + cudaGetErrorString(e_));      \
    } while (0)

}  // namespace

int gnn_param_count() { return layout().total; }

void gnn_features(int n, const std::vector<int> &ei, const std::vector<int> &ej, const std::vector<int32_t> &w,
                  const std::vector<int8_t> &fx, std::vector<float> &out, const std::vector<float> *score) {
    out.assign((size_t)n * kGnnFeat, 0.f);
    std::vector<int> deg(n, 0), fdeg(n, 0), ones(n, 0);
    for (size_t k = 0; k < ei.size(); k++) {
        const int a = ei[k], b = ej[k];
        deg[a]++;
        deg[b]++;
        if (fx[b] < 0) fdeg[a]++;
        if (fx[a] < 0) fdeg[b]++;
        if (fx[b] == 1) ones[a]++;
        if (fx[a] == 1) ones[b]++;
    }
    for (int v = 0; v < n; v++) {
        float *f = &out[(size_t)v * kGnnFeat];
        f[0] = fx[v] < 0;
        f[1] = fx[v] == 0;
        f[2] = fx[v] == 1;
        f[3] = (float)std::abs((double)w[v]) / 10.f;
        f[4] = fdeg[v] / 8.f;
        f[5] = deg[v] / 8.f;
        f[6] = ones[v] / 8.f;
        f[7] = score ? (*score)[v] : 0.f;
    }
}

GnnModel::GnnModel(uint64_t seed) {
    const Layout &L = layout();
    np = L.total;
    std::vector<float> h(np, 0.f);
    uint64_t s = seed;
    auto uni = [&]() {   // SplitMix64 -> [0, 1)
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < kGnnLayers; l++) {
        const int d = din_of(l);
        const double lim = std::sqrt(6.0 / (d + kGnnHidden));   // Glorot-uniform
        for (int i = 0; i < d * kGnnHidden; i++) {
            h[L.W[l] + i] = (float)((2 * uni() - 1) * lim);
            h[L.U[l] + i] = (float)((2 * uni() - 1) * lim * 0.5);
        }
    }
    const double lw = std::sqrt(6.0 / (kGnnHidden + 1));
    for (int j = 0; j < kGnnHidden; j++) h[L.w + j] = (float)((2 * uni() - 1) * lw);
    GNN_CHECK(cudaMalloc(&P, sizeof(float) * np));
    GNN_CHECK(cudaMalloc(&G, sizeof(float) * np));
    GNN_CHECK(cudaMalloc(&Mo, sizeof(float) * np));
    GNN_CHECK(cudaMalloc(&Vo, sizeof(float) * np));
    GNN_CHECK(cudaMemcpy(P, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    GNN_CHECK(cudaMemset(G, 0, sizeof(float) * np));
    GNN_CHECK(cudaMemset(Mo, 0, sizeof(float) * np));
    GNN_CHECK(cudaMemset(Vo, 0, sizeof(float) * np));
}

GnnModel::~GnnModel() {
    for (void *p : {(void *)P, (void *)G, (void *)Mo, (void *)Vo, (void *)rowp, (void *)col, (void *)buf})
        if (p) cudaFree(p);
}

void GnnModel::ensure(int nn) {
    const size_t need = (size_t)nn * (kGnnFeat                               // X0
                                      + kGnnFeat + 2 * kGnnHidden           // M[0..2]
                                      + 2 * kGnnLayers * kGnnHidden         // Z, H
                                      + 4                                   // S, Y, Msk, dS
                                      + 4 * kGnnHidden) + 64;               // dZ, dZb, dX, dP, loss
    if (need > bufcap) {
        if (buf) cudaFree(buf);
        buf = nullptr;
        GNN_CHECK(cudaMalloc(&buf, sizeof(float) * need));
        bufcap = need;
    }
    float *q = buf;
    auto take = [&](size_t k) { float *r = q; q += k; return r; };
    X0 = take((size_t)nn * kGnnFeat);
    for (int l = 0; l < kGnnLayers; l++) M[l] = take((size_t)nn * din_of(l));
    for (int l = 0; l < kGnnLayers; l++) {
        Z[l] = take((size_t)nn * kGnnHidden);
        H[l] = take((size_t)nn * kGnnHidden);
    }
    S = take(nn);
    Y = take(nn);
    Msk = take(nn);
    dS = take(nn);
    dZ = take((size_t)nn * kGnnHidden);
    dZb = take((size_t)nn * kGnnHidden);
    dX = take((size_t)nn * kGnnHidden);
    dP = take((size_t)nn * kGnnHidden);
    loss = take(1);
}

void GnnModel::set_graph(int nn, const std::vector<int> &ei, const std::vector<int> &ej, cudaStream_t s) {
    n = nn;
    std::vector<int> rp(nn + 1, 0), cl(2 * ei.size());
    for (size_t k = 0; k < ei.size(); k++) {
        rp[ei[k] + 1]++;
        rp[ej[k] + 1]++;
    }
    for (int v = 0; v < nn; v++) rp[v + 1] += rp[v];
    std::vector<int> pos(rp.begin(), rp.end() - 1);
    for (size_t k = 0; k < ei.size(); k++) {
        cl[pos[ei[k]]++] = ej[k];
        cl[pos[ej[k]]++] = ei[k];
    }
    if (nn + 1 > ncap) {
        if (rowp) cudaFree(rowp);
        GNN_CHECK(cudaMalloc(&rowp, sizeof(int) * (nn + 1)));
        ncap = nn + 1;
    }
    if ((int)cl.size() + 1 > ecap) {
        if (col) cudaFree(col);
        GNN_CHECK(cudaMalloc(&col, sizeof(int) * (cl.size() + 1)));
        ecap = (int)cl.size() + 1;
    }
    GNN_CHECK(cudaMemcpyAsync(rowp, rp.data(), sizeof(int) * (nn + 1), cudaMemcpyHostToDevice, s));
    if (!cl.empty()) GNN_CHECK(cudaMemcpyAsync(col, cl.data(), sizeof(int) * cl.size(), cudaMemcpyHostToDevice, s));
    ensure(nn);
    GNN_CHECK(cudaStreamSynchronize(s));
}

void GnnModel::fwd(const float *feats, cudaStream_t s) {
    const Layout &L = layout();
    GNN_CHECK(cudaMemcpyAsync(X0, feats, sizeof(float) * (size_t)n * kGnnFeat, cudaMemcpyHostToDevice, s));
    for (int l = 0; l < kGnnLayers; l++) {
        const float *Hin = l == 0 ? X0 : H[l - 1];
        const int d = din_of(l);
        GNN_CHECK(gnn_gather(n, d, rowp, col, Hin, M[l], s));
        GNN_CHECK(gnn_dense(n, d, kGnnHidden, Hin, M[l], P + L.W[l], P + L.U[l], P + L.b[l], Z[l], H[l], 1, s));
    }
    GNN_CHECK(gnn_dense(n, kGnnHidden, 1, H[kGnnLayers - 1], nullptr, P + L.w, nullptr, P + L.c, S, nullptr, 0, s));
}

void GnnModel::forward(const float *feats, std::vector<float> &scores, cudaStream_t s) {
    fwd(feats, s);
    scores.resize(n);
    GNN_CHECK(cudaMemcpyAsync(scores.data(), S, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    GNN_CHECK(cudaStreamSynchronize(s));
}

float GnnModel::train_step(const float *feats, const float *labels, const float *mask, float lr, cudaStream_t s) {
    const Layout &L = layout();
    double cnt = 0;
    for (int v = 0; v < n; v++) cnt += mask[v];
    const float inv = cnt > 0 ? (float)(1.0 / cnt) : 0.f;
    fwd(feats, s);
    GNN_CHECK(cudaMemcpyAsync(Y, labels, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    GNN_CHECK(cudaMemcpyAsync(Msk, mask, sizeof(float) * n, cudaMemcpyHostToDevice, s));
    GNN_CHECK(cudaMemsetAsync(loss, 0, sizeof(float), s));
    GNN_CHECK(gnn_loss(n, S, Y, Msk, inv, dS, loss, s));
    // head
    GNN_CHECK(gnn_wgrad(n, kGnnHidden, 1, H[kGnnLayers - 1], nullptr, dS, G + L.w, nullptr, s));
    GNN_CHECK(gnn_bgrad(n, 1, dS, G + L.c, s));
    GNN_CHECK(gnn_head_back(n, kGnnHidden, dS, P + L.w, Z[kGnnLayers - 1], dZ, s));
    float *cur = dZ, *nxt = dZb;
    for (int l = kGnnLayers - 1; l >= 0; l--) {
        const float *Hin = l == 0 ? X0 : H[l - 1];
        const int d = din_of(l);
        GNN_CHECK(gnn_wgrad(n, d, kGnnHidden, Hin, M[l], cur, G + L.W[l], G + L.U[l], s));
        GNN_CHECK(gnn_bgrad(n, kGnnHidden, cur, G + L.b[l], s));
        if (l > 0) {
            GNN_CHECK(gnn_xgrad(n, d, kGnnHidden, cur, P + L.W[l], P + L.U[l], dX, dP, s));
            GNN_CHECK(gnn_xgrad_finish(n, d, rowp, col, dX, dP, Z[l - 1], nxt, s));
            std::swap(cur, nxt);
        }
    }
    if (lr > 0) {
        step++;
        GNN_CHECK(gnn_adam(np, P, G, Mo, Vo, lr, step, s));
    }
    float h = 0;
    GNN_CHECK(cudaMemcpyAsync(&h, loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    GNN_CHECK(cudaStreamSynchronize(s));
    return h;
}

void GnnModel::get_params(std::vector<float> &p) const {
    p.resize(np);
    GNN_CHECK(cudaMemcpy(p.data(), P, sizeof(float) * np, cudaMemcpyDeviceToHost));
}

void GnnModel::set_params(const std::vector<float> &p) {
    if ((int)p.size() != np) fail(BBTN_EINVAL, "gnn: wrong parameter count");
    GNN_CHECK(cudaMemcpy(P, p.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    step = 0;
    GNN_CHECK(cudaMemset(Mo, 0, sizeof(float) * np));
    GNN_CHECK(cudaMemset(Vo, 0, sizeof(float) * np));
}

void GnnModel::get_grads(std::vector<float> &g) const {
    g.resize(np);
    GNN_CHECK(cudaMemcpy(g.data(), G, sizeof(float) * np, cudaMemcpyDeviceToHost));
}

}  // namespace bbtn

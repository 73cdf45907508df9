// K7: graph neural network scorer (message passing, 3 layers, hidden 64, fp32)
// with hand-written forward, backward and Adam kernels. It scores vertices of a
// branch-and-bound sub-problem (the paper's discussion proposes learned branching
// policies in place of the myopic heuristics); the solver uses the scores to order
// branches so that a good incumbent appears early.
//
// Layer l (l = 1..3):  Z_l = H_{l-1} W_l + (A H_{l-1}) U_l + b_l,  H_l = relu(Z_l)
// Head:                s = H_3 w + c      (one logit per vertex)
// Loss:                mean over masked vertices of softplus(s) - y s  (labels y in {0,1})
// A is the (symmetric) adjacency matrix, applied through CSR lists.
#include <cuda_runtime.h>

#include "gnn.h"

namespace bbtn {

namespace {

constexpr int kT = 256;

// M[v, :] = sum over neighbours u of H[u, :]   (one warp per vertex, lanes over features)
__global__ void k_gather(int n, int d, const int *rowp, const int *col, const float *H, float *M) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    for (int f = lane; f < d; f += 32) {
        float acc = 0.f;
        for (int e = rowp[w]; e < rowp[w + 1]; e++) acc += H[(size_t)col[e] * d + f];
        M[(size_t)w * d + f] = acc;
    }
}

// Z = X W + M U + b (X, M: n x din; W, U: din x dout); H = relu(Z) if relu
__global__ void k_dense(int n, int din, int dout, const float *X, const float *M, const float *W, const float *U,
                        const float *b, float *Z, float *H, int relu) {
    extern __shared__ float sw[];   // W then U, din x dout each
    for (int i = threadIdx.x; i < din * dout; i += blockDim.x) {
        sw[i] = W[i];
        sw[din * dout + i] = U ? U[i] : 0.f;
    }
    __syncthreads();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * dout) return;
    const int v = (int)(idx / dout), j = (int)(idx % dout);
    float acc = b ? b[j] : 0.f;
    for (int i = 0; i < din; i++) {
        acc += X[(size_t)v * din + i] * sw[i * dout + j];
        if (M) acc += M[(size_t)v * din + i] * sw[din * dout + i * dout + j];
    }
    Z[idx] = acc;
    if (H) H[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// dS = (sigmoid(s) - y) * mask / count ; loss partial sums
__global__ void k_loss(int n, const float *s, const float *y, const float *mask, float inv_count, float *dS,
                       float *loss) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (v < n) {
        const float m = mask[v], z = s[v];
        const float sp = z > 0 ? z + log1pf(expf(-z)) : log1pf(expf(z));   // softplus
        l = m * (sp - y[v] * z) * inv_count;
        dS[v] = m * (1.f / (1.f + expf(-z)) - y[v]) * inv_count;
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// G (din x dout) = X^T dZ  [+ M^T dZ into GU] ; one block per row i of the weight, threads over j
__global__ void k_wgrad(int n, int din, int dout, const float *X, const float *M, const float *dZ, float *GW,
                        float *GU) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < dout; j += blockDim.x) {
        float a = 0.f, c = 0.f;
        for (int v = 0; v < n; v++) {
            const float g = dZ[(size_t)v * dout + j];
            a += X[(size_t)v * din + i] * g;
            if (M) c += M[(size_t)v * din + i] * g;
        }
        GW[i * dout + j] = a;
        if (GU) GU[i * dout + j] = c;
    }
}

// gb[j] = sum_v dZ[v, j]
__global__ void k_bgrad(int n, int dout, const float *dZ, float *gb) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= dout) return;
    float a = 0.f;
    for (int v = 0; v < n; v++) a += dZ[(size_t)v * dout + j];
    gb[j] = a;
}

// dX = dZ W^T (n x din) ; dP = dZ U^T (n x din, to be gathered through A)
__global__ void k_xgrad(int n, int din, int dout, const float *dZ, const float *W, const float *U, float *dX,
                        float *dP) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * din) return;
    const int v = (int)(idx / din), i = (int)(idx % din);
    float a = 0.f, c = 0.f;
    for (int j = 0; j < dout; j++) {
        const float g = dZ[(size_t)v * dout + j];
        a += g * W[i * dout + j];
        c += g * U[i * dout + j];
    }
    dX[idx] = a;
    dP[idx] = c;
}

// dH = dX + A dP (A symmetric); then through the relu of the layer below: dZ = dH * (Z > 0)
__global__ void k_xgrad_finish(int n, int d, const int *rowp, const int *col, const float *dX, const float *dP,
                               const float *Zbelow, float *dZbelow) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= n) return;
    for (int f = lane; f < d; f += 32) {
        float acc = dX[(size_t)w * d + f];
        for (int e = rowp[w]; e < rowp[w + 1]; e++) acc += dP[(size_t)col[e] * d + f];
        dZbelow[(size_t)w * d + f] = Zbelow[(size_t)w * d + f] > 0.f ? acc : 0.f;
    }
}

// dZ3 = dS w^T masked by relu(Z3) ; also gw = H3^T dS, gc = sum dS
__global__ void k_head_back(int n, int d, const float *dS, const float *w, const float *Z3, float *dZ3) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)n * d) return;
    const int v = (int)(idx / d), j = (int)(idx % d);
    dZ3[idx] = Z3[idx] > 0.f ? dS[v] * w[j] : 0.f;
}

__global__ void k_adam(int np, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    m[i] = b1 * m[i] + (1.f - b1) * gi;
    v[i] = b2 * v[i] + (1.f - b2) * gi * gi;
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

inline unsigned nblk(size_t n, int t = kT) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t gnn_gather(int n, int d, const int *rowp, const int *col, const float *H, float *M, cudaStream_t s) {
    k_gather<<<nblk((size_t)n * 32), kT, 0, s>>>(n, d, rowp, col, H, M);
    return cudaGetLastError();
}

cudaError_t gnn_dense(int n, int din, int dout, const float *X, const float *M, const float *W, const float *U,
                      const float *b, float *Z, float *H, int relu, cudaStream_t s) {
    const size_t smem = 2 * (size_t)din * dout * sizeof(float);
    k_dense<<<nblk((size_t)n * dout), kT, smem, s>>>(n, din, dout, X, M, W, U, b, Z, H, relu);
    return cudaGetLastError();
}

cudaError_t gnn_loss(int n, const float *sc, const float *y, const float *mask, float inv_count, float *dS,
                     float *loss, cudaStream_t s) {
    k_loss<<<nblk(n), kT, 0, s>>>(n, sc, y, mask, inv_count, dS, loss);
    return cudaGetLastError();
}

cudaError_t gnn_wgrad(int n, int din, int dout, const float *X, const float *M, const float *dZ, float *GW, float *GU,
                      cudaStream_t s) {
    k_wgrad<<<din, 64, 0, s>>>(n, din, dout, X, M, dZ, GW, GU);
    return cudaGetLastError();
}

cudaError_t gnn_bgrad(int n, int dout, const float *dZ, float *gb, cudaStream_t s) {
    k_bgrad<<<nblk(dout, 64), 64, 0, s>>>(n, dout, dZ, gb);
    return cudaGetLastError();
}

cudaError_t gnn_xgrad(int n, int din, int dout, const float *dZ, const float *W, const float *U, float *dX, float *dP,
                      cudaStream_t s) {
    k_xgrad<<<nblk((size_t)n * din), kT, 0, s>>>(n, din, dout, dZ, W, U, dX, dP);
    return cudaGetLastError();
}

cudaError_t gnn_xgrad_finish(int n, int d, const int *rowp, const int *col, const float *dX, const float *dP,
                             const float *Zbelow, float *dZbelow, cudaStream_t s) {
    k_xgrad_finish<<<nblk((size_t)n * 32), kT, 0, s>>>(n, d, rowp, col, dX, dP, Zbelow, dZbelow);
    return cudaGetLastError();
}

cudaError_t gnn_head_back(int n, int d, const float *dS, const float *w, const float *Z3, float *dZ3, cudaStream_t s) {
    k_head_back<<<nblk((size_t)n * d), kT, 0, s>>>(n, d, dS, w, Z3, dZ3);
    return cudaGetLastError();
}

cudaError_t gnn_adam(int np, float *p, const float *g, float *m, float *v, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    for (int i = 0; i < step; i++) { c1 *= b1; c2 *= b2; }
    k_adam<<<nblk(np), kT, 0, s>>>(np, p, g, m, v, lr, b1, b2, 1e-8f, 1.f - c1, 1.f - c2);
    return cudaGetLastError();
}

}  // namespace bbtn

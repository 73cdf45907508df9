// Graph neural network branch scorer: kernels (gnn.cu) and the model (gnn_model.cpp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace bbtn {

constexpr int kGnnFeat = 8;     // input features per vertex
constexpr int kGnnHidden = 64;  // hidden width
constexpr int kGnnLayers = 3;
constexpr int kGnnBranchCandidates = 8;    // seeds a branch scorer chooses among (at least)

cudaError_t gnn_gather(int n, int d, const int *rowp, const int *col, const float *H, float *M, cudaStream_t s);
cudaError_t gnn_dense(int n, int din, int dout, const float *X, const float *M, const float *W, const float *U,
                      const float *b, float *Z, float *H, int relu, cudaStream_t s);
cudaError_t gnn_loss(int n, const float *sc, const float *y, const float *mask, float inv_count, float *dS,
                     float *loss, cudaStream_t s);
cudaError_t gnn_wgrad(int n, int din, int dout, const float *X, const float *M, const float *dZ, float *GW, float *GU,
                      cudaStream_t s);
cudaError_t gnn_bgrad(int n, int dout, const float *dZ, float *gb, cudaStream_t s);
cudaError_t gnn_xgrad(int n, int din, int dout, const float *dZ, const float *W, const float *U, float *dX, float *dP,
                      cudaStream_t s);
cudaError_t gnn_xgrad_finish(int n, int d, const int *rowp, const int *col, const float *dX, const float *dP,
                             const float *Zbelow, float *dZbelow, cudaStream_t s);
cudaError_t gnn_head_back(int n, int d, const float *dS, const float *w, const float *Z3, float *dZ3, cudaStream_t s);
cudaError_t gnn_adam(int np, float *p, const float *g, float *m, float *v, float lr, int step, cudaStream_t s);

// Parameter layout (flat fp32): per layer l: W_l (din x 64), U_l (din x 64), b_l (64),
// din = 8 for l = 1 else 64; then the head w (64) and c (1).
int gnn_param_count();

// Per-vertex input features of a sub-problem: fx[v] = -1 free, 0 / 1 fixed; w:
// vertex weights (MWIS) or |2 h_v| (spin glass); score: the variable's share of the
// overflow (0..1; NULL = 0). Row-major n x kGnnFeat.
void gnn_features(int n, const std::vector<int> &ei, const std::vector<int> &ej, const std::vector<int32_t> &w,
                  const std::vector<int8_t> &fx, std::vector<float> &out, const std::vector<float> *score = nullptr);

class GnnModel {
  public:
    explicit GnnModel(uint64_t seed);
    ~GnnModel();
    void set_graph(int n, const std::vector<int> &ei, const std::vector<int> &ej, cudaStream_t s);
    // logits for every vertex (host vector)
    void forward(const float *feats, std::vector<float> &scores, cudaStream_t s);
    // one Adam step on the masked binary cross-entropy; returns the loss. With
    // lr <= 0 only the gradients are computed (grads() reads them back).
    float train_step(const float *feats, const float *labels, const float *mask, float lr, cudaStream_t s);
    void get_params(std::vector<float> &p) const;
    void set_params(const std::vector<float> &p);
    void get_grads(std::vector<float> &g) const;
    int n = 0;

  private:
    void ensure(int n);
    void fwd(const float *feats_dev, cudaStream_t s);
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;   // params, grads, Adam moments
    int np = 0, step = 0;
    int *rowp = nullptr, *col = nullptr;
    int ncap = 0, ecap = 0;
    float *buf = nullptr;      // activations and temporaries
    size_t bufcap = 0;
    // activation views inside buf
    float *X0 = nullptr, *M[kGnnLayers] = {}, *Z[kGnnLayers] = {}, *H[kGnnLayers] = {}, *S = nullptr,
          *Y = nullptr, *Msk = nullptr, *dS = nullptr, *dZ = nullptr, *dZb = nullptr, *dX = nullptr, *dP = nullptr,
          *loss = nullptr;
};

}  // namespace bbtn

// prop.cuh -- declarations shared by the proposal network's training and inference code.
#pragma once

#include <vector>

#include "hgm_internal.cuh"

namespace hgm {

constexpr int kPropHidden = 128;
constexpr uint32_t kPropMagic = 0x50524f50u;   // "PROP"

// Flat FP32 parameter vector: W1 [H x dp] (d_in used), b1, W2 [H x H], b2, w3, b3 (padded to 4).
struct PropLayout {
    int F = 0, d_in = 0, dp = 0;
    int64_t o_W1 = 0, o_b1 = 0, o_W2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0, n = 0, n_logical = 0;
};

// Per-batch activations and scratch of the training kernels.
struct PropTrain {
    void *buf = nullptr;
    int cap = 0;
    float *z1, *h1, *z2, *h2, *dz2, *dh1, *t_a, *t_b, *spare, *z3, *dz3, *lossv, *loss, *xt, *w2t;
    int *status;
    cudaError_t ensure(const PropLayout &L, int B);
};

PropLayout prop_layout(int F);
void prop_pack(const PropLayout &L, const float *logical, std::vector<float> &flat);
void prop_unpack(const PropLayout &L, const float *flat, float *logical);
void prop_init(const PropLayout &L, uint64_t seed, std::vector<float> &logical);
cudaError_t prop_forward(const PropLayout &L, const float *theta, PropTrain &w, const float *X, int ldx, int B,
                         cudaStream_t st);
cudaError_t prop_backward(const PropLayout &L, const float *theta, PropTrain &w, const float *X, int ldx,
                          const float *y, int B, float *grad, cudaStream_t st);
cudaError_t prop_adam(const PropLayout &L, float *theta, const float *grad, float *m, float *v, int64_t t, float lr,
                      cudaStream_t st);

}  // namespace hgm

struct hgm_prop;
void prop_free(hgm_prop *p);   // device buffers of a proposal handle (prop_api.cu)

struct hgm_prop {
    uint32_t magic;
    hgm::PropLayout L;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // device, L.n floats each
    int64_t step = 0;
    hgm::PropTrain train;
};

// k_prop.cu -- the candidate-proposal network: training (forward, backward, Adam) and weights.
//
// Not part of the paper: a small MLP layered on the exact method that scores each
// window candidate so that only the best `keep` enter the recursion (the pruned
// form; the exact recursion stays its fallback and the yardstick of its recall and energy gap). Architecture:
//   x = [f_i, f'_j, dx/100, dy/100, dt/w]  (d_in = 2F + 3)
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2)  (128 each),  z3 = w3.h2 + b3,  score = sigmoid(z3)
// trained with binary cross-entropy on labels produced by the exact recursion.
//
// Every contraction (the two forward layers, and dW2, dH1, dW1 in the backward
// pass) runs on the tensor cores through the BF16 row-product kernel (FP32
// accumulation); weights, gradients and Adam moments are FP32 master copies.
// Elementwise steps, column sums and the last layer (a 128-long dot product per
// sample) are plain SIMT kernels.
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "hgm_internal.cuh"
#include "prop.cuh"

namespace hgm {
namespace {

constexpr int H = kPropHidden;

__global__ void relu_copy_kernel(const float *__restrict__ z, float *__restrict__ h, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        h[k] = fmaxf(z[k], 0.0f);
}

// z3[b] = w3 . h2[b] + b3 (one warp per sample)
__global__ void last_layer_kernel(const float *__restrict__ h2, int B, const float *__restrict__ w3, const float *b3,
                                  float *__restrict__ z3)
{
    const int lane = threadIdx.x & 31;
    for (int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); b < B; b += gridDim.x * (blockDim.x / 32)) {
        float s = 0.0f;
        for (int h = lane; h < H; h += 32) s = fmaf(h2[(int64_t)b * H + h], w3[h], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) z3[b] = s + b3[0];
    }
}

// dz3 = (sigmoid(z3) - y) / B; per-sample loss softplus(z3) - y z3 into lossv
__global__ void loss_grad_kernel(const float *__restrict__ z3, const float *__restrict__ y, int B,
                                 float *__restrict__ dz3, float *__restrict__ lossv)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const float z = z3[b];
        const float sg = 1.0f / (1.0f + expf(-z));
        dz3[b] = (sg - y[b]) / (float)B;
        const float sp = z > 0.0f ? z + log1pf(expf(-z)) : log1pf(expf(z));
        lossv[b] = sp - y[b] * z;
    }
}

// dZ2[b][n] = dz3[b] w3[n] [z2 > 0]
__global__ void dz2_kernel(const float *__restrict__ dz3, const float *__restrict__ w3, const float *__restrict__ z2,
                           int B, float *__restrict__ dz2)
{
    const int64_t n = (int64_t)B * H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dz2[k] = z2[k] > 0.0f ? dz3[k / H] * w3[k % H] : 0.0f;
}

// g[k] = (z[k] > 0) ? g[k] : 0
__global__ void relu_mask_kernel(float *__restrict__ g, const float *__restrict__ z, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (!(z[k] > 0.0f)) g[k] = 0.0f;
}

// out[c] = sum_b X[b][c] (column sums, fixed order), optionally out[c] = sum_b X[b][c] * w[b]
__global__ void colsum_kernel(const float *__restrict__ X, int B, int C, const float *__restrict__ w,
                              float *__restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += w ? X[(int64_t)b * C + c] * w[b] : X[(int64_t)b * C + c];
        out[c] = s;
    }
}

__global__ void sum_kernel(const float *__restrict__ v, int n, float scale, float *__restrict__ out)
{
    __shared__ float part[32];
    float s = 0.0f;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += v[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        *out = t * scale;
    }
}

// out[c][r] = in[r][c] for an R x C row-major matrix (ld_in, ld_out in floats)
__global__ void transpose_kernel(const float *__restrict__ in, int R, int C, int ld_in, float *__restrict__ out,
                                 int ld_out)
{
    __shared__ float tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < R && c < C) ? in[(int64_t)r * ld_in + c] : 0.0f;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (c < C && r < R) out[(int64_t)c * ld_out + r] = tile[threadIdx.x][k];
    }
}

// Adam (bias-corrected) on the flat parameter vector
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.0f - b1) * gk;
        const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

unsigned blocks_for(int64_t n, int per = 256) { return (unsigned)std::min<int64_t>((n + per - 1) / per, 4096); }

cudaError_t transpose(const float *in, int R, int C, int ld_in, float *out, int ld_out, cudaStream_t st)
{
    dim3 grid((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32));
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, R, C, ld_in, out, ld_out);
    return cudaGetLastError();
}

}  // namespace

// ---- parameter layout ------------------------------------------------------------------------
PropLayout prop_layout(int F)
{
    PropLayout L;
    L.F = F;
    L.d_in = 2 * F + 3;
    L.dp = (L.d_in + 3) & ~3;
    L.o_W1 = 0;
    L.o_b1 = L.o_W1 + (int64_t)H * L.dp;
    L.o_W2 = L.o_b1 + H;
    L.o_b2 = L.o_W2 + (int64_t)H * H;
    L.o_w3 = L.o_b2 + H;
    L.o_b3 = L.o_w3 + H;
    L.n = L.o_b3 + 4;
    L.n_logical = (int64_t)H * L.d_in + H + (int64_t)H * H + H + H + 1;
    return L;
}

// logical (W1 [H x d_in], b1, W2, b2, w3, b3) <-> padded device layout
void prop_pack(const PropLayout &L, const float *logical, std::vector<float> &flat)
{
    flat.assign((size_t)L.n, 0.0f);
    const float *p = logical;
    for (int h = 0; h < H; ++h) std::memcpy(&flat[(size_t)(L.o_W1 + (int64_t)h * L.dp)], p + (int64_t)h * L.d_in,
                                            sizeof(float) * (size_t)L.d_in);
    p += (int64_t)H * L.d_in;
    std::memcpy(&flat[(size_t)L.o_b1], p, sizeof(float) * H);
    p += H;
    std::memcpy(&flat[(size_t)L.o_W2], p, sizeof(float) * H * H);
    p += (int64_t)H * H;
    std::memcpy(&flat[(size_t)L.o_b2], p, sizeof(float) * H);
    p += H;
    std::memcpy(&flat[(size_t)L.o_w3], p, sizeof(float) * H);
    p += H;
    flat[(size_t)L.o_b3] = p[0];
}

void prop_unpack(const PropLayout &L, const float *flat, float *logical)
{
    float *p = logical;
    for (int h = 0; h < H; ++h)
        std::memcpy(p + (int64_t)h * L.d_in, flat + L.o_W1 + (int64_t)h * L.dp, sizeof(float) * (size_t)L.d_in);
    p += (int64_t)H * L.d_in;
    std::memcpy(p, flat + L.o_b1, sizeof(float) * H);
    p += H;
    std::memcpy(p, flat + L.o_W2, sizeof(float) * H * H);
    p += (int64_t)H * H;
    std::memcpy(p, flat + L.o_b2, sizeof(float) * H);
    p += H;
    std::memcpy(p, flat + L.o_w3, sizeof(float) * H);
    p += H;
    p[0] = flat[L.o_b3];
}

void prop_init(const PropLayout &L, uint64_t seed, std::vector<float> &logical)
{
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    logical.assign((size_t)L.n_logical, 0.0f);
    float *p = logical.data();
    const double s1 = std::sqrt(2.0 / L.d_in), s2 = std::sqrt(2.0 / H), s3 = std::sqrt(1.0 / H);
    for (int64_t k = 0; k < (int64_t)H * L.d_in; ++k) p[k] = (float)(nd(gen) * s1);
    p += (int64_t)H * L.d_in + H;
    for (int64_t k = 0; k < (int64_t)H * H; ++k) p[k] = (float)(nd(gen) * s2);
    p += (int64_t)H * H + H;
    for (int k = 0; k < H; ++k) p[k] = (float)(nd(gen) * s3);
}

// ---- training workspace -----------------------------------------------------------------------
cudaError_t PropTrain::ensure(const PropLayout &L, int B)
{
    if (B <= cap && buf) return cudaSuccess;
    if (buf) cudaFree(buf);
    buf = nullptr;
    cap = 0;
    const int64_t BH = (int64_t)B * H;
    size_t floats = (size_t)(BH * 9 + (int64_t)B * 4 + (int64_t)L.dp * B + (int64_t)H * H + 64);
    cudaError_t e = cudaMalloc(&buf, floats * sizeof(float));
    if (e != cudaSuccess) return e;
    float *q = static_cast<float *>(buf);
    auto take = [&](int64_t n) { float *r = q; q += (n + 3) & ~int64_t(3); return r; };
    z1 = take(BH); h1 = take(BH); z2 = take(BH); h2 = take(BH);
    dz2 = take(BH); dh1 = take(BH); t_a = take(BH); t_b = take(BH); spare = take(BH);
    z3 = take(B); dz3 = take(B); lossv = take(B); loss = take(4);
    xt = take((int64_t)L.dp * B);
    w2t = take((int64_t)H * H);
    status = reinterpret_cast<int *>(take(4));
    cap = B;
    return cudaMemset(status, 0, sizeof(int));
}

// forward: Z1, H1, Z2, H2, z3 for X [B x d_in] (row stride ldx)
cudaError_t prop_forward(const PropLayout &L, const float *theta, PropTrain &w, const float *X, int ldx, int B,
                         cudaStream_t st)
{
    cudaError_t e;
    const int64_t BH = (int64_t)B * H;
    if ((e = launch_rowdot_plain(X, B, ldx, theta + L.o_W1, H, L.dp, L.d_in, theta + L.o_b1, w.z1, H, w.status, st)))
        return e;
    relu_copy_kernel<<<blocks_for(BH), 256, 0, st>>>(w.z1, w.h1, BH);
    if ((e = launch_rowdot_plain(w.h1, B, H, theta + L.o_W2, H, H, H, theta + L.o_b2, w.z2, H, w.status, st)))
        return e;
    relu_copy_kernel<<<blocks_for(BH), 256, 0, st>>>(w.z2, w.h2, BH);
    last_layer_kernel<<<blocks_for((int64_t)B * 32), 256, 0, st>>>(w.h2, B, theta + L.o_w3, theta + L.o_b3, w.z3);
    return cudaGetLastError();
}

// backward into grad (padded layout) after prop_forward with labels y; loss (mean) into w.loss[0]
cudaError_t prop_backward(const PropLayout &L, const float *theta, PropTrain &w, const float *X, int ldx,
                          const float *y, int B, float *grad, cudaStream_t st)
{
    cudaError_t e;
    const int64_t BH = (int64_t)B * H;
    if ((e = cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)L.n, st))) return e;
    loss_grad_kernel<<<blocks_for(B), 256, 0, st>>>(w.z3, y, B, w.dz3, w.lossv);
    sum_kernel<<<1, 256, 0, st>>>(w.lossv, B, 1.0f / (float)B, w.loss);
    // last layer
    colsum_kernel<<<1, H, 0, st>>>(w.h2, B, H, w.dz3, grad + L.o_w3);
    sum_kernel<<<1, 256, 0, st>>>(w.dz3, B, 1.0f, grad + L.o_b3);
    // layer 2
    dz2_kernel<<<blocks_for(BH), 256, 0, st>>>(w.dz3, theta + L.o_w3, w.z2, B, w.dz2);
    colsum_kernel<<<1, H, 0, st>>>(w.dz2, B, H, nullptr, grad + L.o_b2);
    if ((e = transpose(w.dz2, B, H, H, w.t_a, B, st))) return e;   // dZ2^T [H x B]
    if ((e = transpose(w.h1, B, H, H, w.t_b, B, st))) return e;    // H1^T  [H x B]
    if ((e = launch_rowdot_plain(w.t_a, H, B, w.t_b, H, B, B, nullptr, grad + L.o_W2, H, w.status, st))) return e;
    if ((e = transpose(theta + L.o_W2, H, H, H, w.w2t, H, st))) return e;   // W2^T
    if ((e = launch_rowdot_plain(w.dz2, B, H, w.w2t, H, H, H, nullptr, w.dh1, H, w.status, st))) return e;
    relu_mask_kernel<<<blocks_for(BH), 256, 0, st>>>(w.dh1, w.z1, BH);   // dZ1
    colsum_kernel<<<1, H, 0, st>>>(w.dh1, B, H, nullptr, grad + L.o_b1);
    if ((e = transpose(w.dh1, B, H, H, w.t_a, B, st))) return e;        // dZ1^T [H x B]
    if ((e = transpose(X, B, L.d_in, ldx, w.xt, B, st))) return e;      // X^T [d_in x B]
    if ((e = launch_rowdot_plain(w.t_a, H, B, w.xt, L.d_in, B, B, nullptr, grad + L.o_W1, L.dp, w.status, st)))
        return e;
    return cudaGetLastError();
}

cudaError_t prop_adam(const PropLayout &L, float *theta, const float *grad, float *m, float *v, int64_t t, float lr,
                      cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)t), c2 = 1.0f - (float)std::pow(0.999, (double)t);
    adam_kernel<<<blocks_for(L.n), 256, 0, st>>>(theta, grad, m, v, L.n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace hgm

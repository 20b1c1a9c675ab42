// k_unary.cu -- kernel (a): the unary look-up table of Sec. 3.3.
//
// U[r][j] = lambda1 * ||A_r - B_j||_2 for every model row r and scene row j
// (Eq. 2, non-dummy branch, with lambda1 of Eq. 1 absorbed). The paper
// pre-computes this S x M table once instead of re-evaluating the distance
// inside every cell of the trellis; here it is one launch per (model set,
// scene), stored row-major with the scene index contiguous so that a model
// point's window [minnode(f0), minnode(f1+1)) is one coalesced segment.
//
// Every output is accumulated in a fixed order: d_k = A_rk - B_jk (FP32),
// s = fma(d_k, d_k, s) for k = 0, 1, ..., then an IEEE square root and an
// FP32 multiply. The value is therefore reproducible bit for bit by any
// IEEE-754 implementation, which makes it usable as the ranking key of the
// top-K candidate cap. Rows are padded with zeros to a multiple of 4
// components; fma(0, 0, s) == s, so padding changes no bit.
//
// Register tile 4 (r) x 4 (j) per thread, 256 threads, 32 x 128 outputs per
// block; operands staged k-major in shared memory so that the inner loop is
// two 16-byte shared loads per 32 FP32 operations.
#include "hgm_internal.cuh"

namespace hgm {
namespace {

constexpr int BR = 32;     // rows (model points) per block
constexpr int BJ = 128;    // columns (scene points) per block
constexpr int KC = 16;     // components per shared-memory stage
constexpr int PAD_A = 4;
constexpr int PAD_B = 4;

__global__ void __launch_bounds__(256) unary_kernel(const float *__restrict__ A, int R,
                                                    const float *__restrict__ B, int S, int F,
                                                    float lambda1, float *__restrict__ U, int64_t ldu,
                                                    bool vec_store)
{
    __shared__ __align__(16) float sA[KC][BR + PAD_A];
    __shared__ __align__(16) float sB[KC][BJ + PAD_B];
    const int tid = threadIdx.x;
    const int tx = tid & 31;          // column group: j = j0 + 4*tx + {0..3}
    const int ty = tid >> 5;          // row group:    r = r0 + 4*ty + {0..3}
    const int r0 = blockIdx.y * BR;
    const int64_t j0 = (int64_t)blockIdx.x * BJ;

    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;

    for (int k0 = 0; k0 < F; k0 += KC) {
        // stage A: 32 rows x 16 components, 2 per thread
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int e = tid + 256 * q;
            int r = e / KC, k = e % KC;
            float v = 0.0f;
            if (r0 + r < R && k0 + k < F) v = A[(int64_t)(r0 + r) * F + k0 + k];
            sA[k][r] = v;
        }
        // stage B: 128 rows x 16 components, 8 per thread
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            int e = tid + 256 * q;
            int j = e / KC, k = e % KC;
            float v = 0.0f;
            if (j0 + j < S && k0 + k < F) v = B[(j0 + j) * F + k0 + k];
            sB[k][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KC; ++k) {
            float4 av = *reinterpret_cast<const float4 *>(&sA[k][4 * ty]);
            float4 bv = *reinterpret_cast<const float4 *>(&sB[k][4 * tx]);
            float a4[4] = {av.x, av.y, av.z, av.w};
            float b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    float d = __fsub_rn(a4[a], b4[b]);
                    acc[a][b] = __fmaf_rn(d, d, acc[a][b]);
                }
        }
        __syncthreads();
    }
    // Components past F were staged as zeros: fma(0,0,s) = s keeps the order exact.
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int r = r0 + 4 * ty + a;
        if (r >= R) continue;
        int64_t j = j0 + 4 * tx;
        float o[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) o[b] = __fmul_rn(lambda1, __fsqrt_rn(acc[a][b]));
        float *row = U + (int64_t)r * ldu;
        if (vec_store && j + 3 < S) {
            *reinterpret_cast<float4 *>(row + j) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (j + b < S) row[j + b] = o[b];
        }
    }
}

}  // namespace

cudaError_t launch_unary(const float *A, int R, const float *B, int S, int F, float lambda1, float *U,
                         int ldu, cudaStream_t st)
{
    if (R <= 0 || S <= 0) return cudaSuccess;
    dim3 grid((unsigned)((S + BJ - 1) / BJ), (unsigned)((R + BR - 1) / BR));
    prof_begin(kProfUnary, st);
    const bool vec_store = ((reinterpret_cast<uintptr_t>(U) & 15) == 0) && ((ldu & 3) == 0);
    unary_kernel<<<grid, 256, 0, st>>>(A, R, B, S, F, lambda1, U, (int64_t)ldu, vec_store);
    prof_end(kProfUnary, st);
    return cudaGetLastError();
}

cudaError_t preload_unary()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, unary_kernel);
}

}  // namespace hgm

// k_rowdot.cu -- BF16 tensor-core row products: dot(x_r, w_c) for every row r of X and c of W.
//
// Used for (1) the unary table of Sec. 3.3 in the precision mode: U = lambda1 *
// sqrt(max(0, |x~|^2 + |w~|^2 - 2 x~.w~)), x~, w~ the BF16-rounded descriptors
// and every product accumulated in FP32 (the expansion of the Euclidean norm of
// Eq. 2 as a contraction), and (2) plain products X W^T (+ bias), e.g. the first
// layer of the proposal network applied once per point.
//
// A CTA owns 128 rows of X at a time (MMA M = 128), stages them once as BF16 in
// shared memory, and sweeps the rows of W in tiles of 128 (MMA N = 128): K/16
// tcgen05.mma (kind::f16) accumulate the 128 x 128 FP32 tile in tensor memory,
// then each warp reads its 32 rows back (tcgen05.ld) and applies the epilogue.
// Two CTAs share an SM (91 KB of shared memory and 128 TMEM columns each).
#include "hgm_internal.cuh"
#include "tc05.cuh"

namespace hgm {
namespace {

constexpr int TM = 128, TN = 128;
constexpr uint32_t kLBO = 128;
constexpr uint32_t kPolls = 1u << 26;   // bounded wait for the tensor core (~0.1 s)

enum Mode { kDist = 0, kPlain = 1 };

// Squared norm of the BF16-rounded row (FP32, components in order).
__global__ void bf16_sqnorm_kernel(const float *__restrict__ X, int64_t n, int ld, int F, float *__restrict__ out)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const float *x = X + r * ld;
        float s = 0.0f;
        for (int k = 0; k < F; ++k) {
            const float v = __bfloat162float(__float2bfloat16_rn(x[k]));
            s = fmaf(v, v, s);
        }
        out[r] = s;
    }
}

// Stages rows [r0, r0+128) x components [k0, k0+K) of a row-major FP32 matrix
// (ld floats per row, F valid components) as BF16 in the canonical K-major
// layout. vec: rows are 16-byte aligned (base and ld), so float4 loads are legal.
__device__ __forceinline__ void stage_rows(unsigned char *dst, const float *__restrict__ X, int64_t nrows, int ld,
                                           int F, int64_t r0, int k0, int K, uint32_t sbo, bool vec, int tid, int nt)
{
    const int chunks = K / 8;
    for (int e = tid; e < TM * chunks; e += nt) {
        const int r = e / chunks, kl = (e % chunks) * 8, k = k0 + kl;
        float v[8];
        const int64_t row = r0 + r;
        if (vec && row < nrows && k + 8 <= F) {
            const float4 *p = reinterpret_cast<const float4 *>(X + row * ld + k);
            const float4 a = p[0], b = p[1];
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (row < nrows && k + q < F) ? X[row * ld + k + q] : 0.0f;
        }
        __align__(16) __nv_bfloat162 h[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
        *reinterpret_cast<uint4 *>(dst + tc05::kmajor_offset(r, kl, kLBO, sbo)) = *reinterpret_cast<uint4 *>(h);
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) rowdot_kernel(const float *__restrict__ X, int64_t nrows, int ldx, bool xvec,
                                                     const float *__restrict__ W, int ncols, int ldw, bool wvec, int F,
                                                     int K, const float *__restrict__ xnorm,
                                                     const float *__restrict__ wnorm, float lambda1,
                                                     const float *__restrict__ bias, float *__restrict__ out,
                                                     int64_t ldo, int *__restrict__ status)
{
    // K is the staged chunk (<= KC); the F components are covered in ceil(F / K) chunks
    extern __shared__ __align__(128) unsigned char smem[];
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    unsigned char *sA = smem;
    unsigned char *sB = smem + (size_t)TM * K * 2;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tc05::tmem_alloc<TN>(&tslot);
    if (tid == 0) {
        tc05::mbar_init(&mbar, 1);
        bad = 0;
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t tlane = taddr + ((uint32_t)(32 * warp) << 16);
    constexpr uint32_t idesc = tc05::idesc_bf16_f32(TM, TN);
    uint32_t phase = 0;
    const int64_t ntiles = (nrows + TM - 1) / TM;
    const int nchunk = (F + K - 1) / K;
    for (int64_t tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
        const int64_t r0 = tile * TM;
        if (nchunk == 1) stage_rows(sA, X, nrows, ldx, F, r0, 0, K, sbo, xvec, tid, 128);
        const int64_t row = r0 + 32 * warp + lane;
        const float xn = (MODE == kDist && row < nrows) ? xnorm[row] : 0.0f;
        for (int c0 = 0; c0 < ncols; c0 += TN) {
            for (int ch = 0; ch < nchunk && !bad; ++ch) {
                if (nchunk > 1) stage_rows(sA, X, nrows, ldx, F, r0, ch * K, K, sbo, xvec, tid, 128);
                stage_rows(sB, W, ncols, ldw, F, c0, ch * K, K, sbo, wvec, tid, 128);
                tc05::fence_proxy_async_smem();
                tc05::fence_before_sync();
                __syncthreads();
                tc05::fence_after_sync();
                if (tid == 0) {
                    const uint32_t a0 = tc05::smem_u32(sA), b0 = tc05::smem_u32(sB);
                    for (int ks = 0; ks < K / 16; ++ks)
                        tc05::mma_bf16(taddr, tc05::smem_desc(a0 + ks * 2 * kLBO, kLBO, sbo),
                                       tc05::smem_desc(b0 + ks * 2 * kLBO, kLBO, sbo), idesc, ch > 0 || ks > 0);
                    tc05::mma_commit(&mbar);
                }
                if (!tc05::mbar_wait(&mbar, phase, kPolls)) {
                    if (lane == 0) { atomicExch(status, 1); bad = 1; }
                }
                phase ^= 1u;
                tc05::fence_before_sync();
                __syncthreads();   // the chunk's operands are consumed: sA / sB may be restaged
                tc05::fence_after_sync();
            }
            if (!bad) {
                for (int cc = 0; cc < TN && c0 + cc < ncols; cc += 32) {
                    float v[32];
                    tc05::tmem_ld32(tlane + (uint32_t)cc, v);
                    if (row < nrows) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int c = c0 + cc + j;
                            if (c < ncols) {
                                if (MODE == kDist) {
                                    const float d2 = fmaxf(xn + wnorm[c] - 2.0f * v[j], 0.0f);
                                    out[(int64_t)c * ldo + row] = lambda1 * sqrtf(d2);
                                } else {
                                    out[row * ldo + c] = v[j] + (bias ? bias[c] : 0.0f);
                                }
                            }
                        }
                    }
                }
            }
            tc05::fence_before_sync();
            __syncthreads();   // TMEM and sB are free again
            tc05::fence_after_sync();
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc<TN>(taddr);
}

constexpr int KC = 256;    // largest K staged at once (A + B tiles: 2 x 128 x 256 x 2 B = 128 KB)

bool aligned16(const void *p, int ld) { return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld & 3) == 0); }

template <int MODE>
cudaError_t launch_rowdot(const float *X, int64_t nrows, int ldx, const float *W, int ncols, int ldw, int F,
                          const float *xnorm, const float *wnorm, float lambda1, const float *bias, float *out,
                          int64_t ldo, int *status, cudaStream_t st)
{
    if (nrows <= 0 || ncols <= 0) return cudaSuccess;
    const int Kfull = (F + 15) / 16 * 16;
    const int K = Kfull <= KC ? Kfull : 128;   // one chunk when it fits, else chunks of 128
    const size_t smem = (size_t)(TM + TN) * K * 2;
    auto kern = rowdot_kernel<MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);   // 4 x 128 TMEM columns = the SM's 512
    int64_t ntiles = (nrows + TM - 1) / TM;
    int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    kern<<<(unsigned)grid, 128, smem, st>>>(X, nrows, ldx, aligned16(X, ldx), W, ncols, ldw, aligned16(W, ldw), F, K,
                                           xnorm, wnorm, lambda1, bias, out, ldo, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sqnorm_bf16(const float *X, int64_t n, int ld, int F, float *out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535);
    bf16_sqnorm_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, n, ld, F, out);
    return cudaGetLastError();
}

cudaError_t launch_unary_bf16(const float *model, int R, const float *scene, int S, int F, int ld,
                              const float *mnorm, const float *snorm, float lambda1, float *U, int64_t ldu,
                              int *status, cudaStream_t st)
{
    prof_begin(kProfUnary, st);
    cudaError_t e = launch_rowdot<kDist>(scene, S, ld, model, R, ld, F, snorm, mnorm, lambda1, nullptr, U, ldu, status,
                                         st);
    prof_end(kProfUnary, st);
    return e;
}

cudaError_t launch_rowdot_plain(const float *X, int64_t nrows, int ldx, const float *W, int ncols, int ldw, int F,
                                const float *bias, float *Y, int64_t ldy, int *status, cudaStream_t st)
{
    return launch_rowdot<kPlain>(X, nrows, ldx, W, ncols, ldw, F, nullptr, nullptr, 0.0f, bias, Y, ldy, status, st);
}

}  // namespace hgm

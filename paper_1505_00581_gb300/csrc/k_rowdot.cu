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
#include <cuda.h>            // CUtensorMap and its enums (types only: the encoder is fetched at run time)
#include <cudaTypedefs.h>    // PFN_cuTensorMapEncodeTiled

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

// ---- the precision mode's unary table with TMA-staged operands ---------------------------------------------
//
// Both operands are first written once as BF16 rows of Kp = F rounded up to 16 components (zeros after F),
// so that the tensor memory accelerator can copy them into shared memory as they are: per 128-row tile and
// 16-byte chunk k8 of K, one cp.async.bulk.tensor box of 8 components x 128 rows lands 128 rows x 16 bytes
// contiguously at k8 x 2048 bytes -- the canonical no-swizzle K-major layout with a K-direction core-matrix
// stride (LBO) of 2048 bytes and a row-group stride (SBO) of 128 bytes. Every box starts at an inner
// coordinate that is a multiple of 8 components (16 bytes); rows past the end of a matrix arrive as zeros.
// A CTA owns 128 scene rows (loaded once) and sweeps the model rows in tiles of 128: one thread issues the
// B tile's boxes on an mbarrier with the expected byte count, waits, issues the MMAs and commits; the 128
// threads read the accumulator (thread = scene row) and write U. Two CTAs share an SM, so one's epilogue
// overlaps the other's copies and MMAs.

constexpr uint32_t kTmaLBO = 2048, kTmaSBO = 128;

__global__ void to_bf16_kernel(const float *__restrict__ X, int64_t n, int ld, int F, int Kp,
                               __nv_bfloat16 *__restrict__ out)
{
    const int64_t total = n * (Kp / 2);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / (Kp / 2);
        const int k = (int)(e - r * (Kp / 2)) * 2;
        const float a = k < F ? X[r * ld + k] : 0.0f, b = k + 1 < F ? X[r * ld + k + 1] : 0.0f;
        reinterpret_cast<__nv_bfloat162 *>(out)[e] = __floats2bfloat162_rn(a, b);
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc05::smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tmap, int x, int y, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(tc05::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(tc05::smem_u32(mbar))
        : "memory");
}

__global__ void __launch_bounds__(128) unary_tma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmB, int64_t S, int R,
                                                        int Kp, const float *__restrict__ snorm,
                                                        const float *__restrict__ mnorm, float lambda1,
                                                        float *__restrict__ U, int64_t ldu, int mrows_per_cta,
                                                        int *__restrict__ status)
{
    // the tiles start on a 1024-byte boundary of the shared window (TMA destinations want 128), whatever the
    // placement of the dynamic array after the static variables: the launch asks for 1024 bytes more
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sA = smem_raw + ((1024u - (tc05::smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *sB = sA + (size_t)TM * Kp * 2;
    __shared__ uint64_t tma_bar, mma_bar;
    __shared__ uint32_t tslot;
    __shared__ float wn[TN];
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc05::tmem_alloc<TN>(&tslot);
    if (tid == 0) {
        tc05::mbar_init(&tma_bar, 1);
        tc05::mbar_init(&mma_bar, 1);
        bad = 0;
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t taddr = tslot;
    const uint32_t tlane = taddr + ((uint32_t)(32 * warp) << 16);
    constexpr uint32_t idesc = tc05::idesc_bf16_f32(TM, TN);
    const int nk8 = Kp / 8;
    const uint32_t tile_bytes = (uint32_t)TM * Kp * 2;
    uint32_t tphase = 0, mphase = 0;
    const int64_t ntiles = (S + TM - 1) / TM;
    // this CTA's model rows: [m_lo, m_hi) of the grid's y dimension
    const int m_lo = (int)blockIdx.y * mrows_per_cta, m_hi = min(R, m_lo + mrows_per_cta);
    for (int64_t tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x) {
        const int64_t r0 = tile * TM;
        const int64_t row = r0 + tid;
        const float xn = row < S ? snorm[row] : 0.0f;
        for (int m0 = m_lo; m0 < m_hi && !bad; m0 += TN) {
            if (tid == 0) {
                // sA and sB are free: the previous tile's MMAs completed (mma_bar) before the last barrier
                mbar_expect_tx(&tma_bar, m0 == m_lo ? 2 * tile_bytes : tile_bytes);
                if (m0 == m_lo)
                    for (int k8 = 0; k8 < nk8; ++k8) tma_load_2d(sA + (size_t)k8 * kTmaLBO, &tmA, 8 * k8, (int)r0, &tma_bar);
                for (int k8 = 0; k8 < nk8; ++k8) tma_load_2d(sB + (size_t)k8 * kTmaLBO, &tmB, 8 * k8, m0, &tma_bar);
            }
            wn[tid] = m0 + tid < m_hi ? mnorm[m0 + tid] : 0.0f;
            if (tid == 0) {
                if (tc05::mbar_wait(&tma_bar, tphase, kPolls)) {
                    tc05::fence_after_sync();
                    const uint32_t a0 = tc05::smem_u32(sA), b0 = tc05::smem_u32(sB);
                    for (int ks = 0; ks < Kp / 16; ++ks)
                        tc05::mma_bf16(taddr, tc05::smem_desc(a0 + ks * 2 * kTmaLBO, kTmaLBO, kTmaSBO),
                                       tc05::smem_desc(b0 + ks * 2 * kTmaLBO, kTmaLBO, kTmaSBO), idesc, ks > 0);
                    tc05::mma_commit(&mma_bar);
                } else {
                    // give the copies in flight a second bounded wait before the CTA leaves
                    tc05::mbar_wait(&tma_bar, tphase, kPolls);
                    if (status) atomicExch(status, 1);
                    bad = 1;
                }
            }
            tphase ^= 1u;
            __syncthreads();   // wn is written; bad is seen by every thread
            if (bad) break;
            if (!tc05::mbar_wait(&mma_bar, mphase, kPolls)) {
                if (status) atomicExch(status, 1);
                bad = 1;
            }
            mphase ^= 1u;
            tc05::fence_after_sync();
            if (!bad) {
                for (int cc = 0; cc < TN && m0 + cc < m_hi; cc += 32) {
                    float v[32];
                    tc05::tmem_ld32(tlane + (uint32_t)cc, v);
                    if (row < S) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int c = m0 + cc + j;
                            if (c < m_hi) {
                                const float d2 = fmaxf(xn + wn[cc + j] - 2.0f * v[j], 0.0f);
                                U[(int64_t)c * ldu + row] = lambda1 * sqrtf(d2);
                            }
                        }
                    }
                }
            }
            tc05::fence_before_sync();
            __syncthreads();   // TMEM, sB and wn are free again
            tc05::fence_after_sync();
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc<TN>(taddr);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D tensor map of n BF16 rows of Kp components, boxes of 8 components x 128 rows.
bool encode_rows(CUtensorMap *tm, const __nv_bfloat16 *base, int64_t n, int Kp)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)TM};
    const cuuint32_t elem[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

size_t unary_bf16_scratch_bytes(int R, int64_t S, int F)
{
    const int64_t Kp = (F + 15) / 16 * 16;
    return (size_t)((R + 255) / 256 * 256 + (S + 255) / 256 * 256) * (size_t)Kp * 2;
}

cudaError_t launch_unary_bf16(const float *model, int R, const float *scene, int S, int F, int ld,
                              const float *mnorm, const float *snorm, float lambda1, float *U, int64_t ldu,
                              int *status, void *scratch, size_t scratch_bytes, cudaStream_t st)
{
    if (R <= 0 || S <= 0) return cudaSuccess;
    prof_begin(kProfUnary, st);
    const int Kp = (F + 15) / 16 * 16;
    cudaError_t e = cudaSuccess;
    CUtensorMap tmA, tmB;
    __nv_bfloat16 *mb = static_cast<__nv_bfloat16 *>(scratch);
    __nv_bfloat16 *sb = mb + (size_t)(R + 255) / 256 * 256 * Kp;
    if (Kp <= KC && scratch && scratch_bytes >= unary_bf16_scratch_bytes(R, S, F) &&
        encode_rows(&tmA, sb, S, Kp) && encode_rows(&tmB, mb, R, Kp)) {
        // BF16 copies of both operands, then the TMA-staged contraction
        const int64_t bm = std::min<int64_t>(((int64_t)R * Kp / 2 + 255) / 256, 65536);
        const int64_t bs = std::min<int64_t>(((int64_t)S * Kp / 2 + 255) / 256, 65536);
        to_bf16_kernel<<<(unsigned)bm, 256, 0, st>>>(model, R, ld, F, Kp, mb);
        to_bf16_kernel<<<(unsigned)bs, 256, 0, st>>>(scene, S, ld, F, Kp, sb);
        const size_t smem = (size_t)2 * TM * Kp * 2 + 1024;
        e = cudaFuncSetAttribute(unary_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 0, per_sm = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, unary_tma_kernel, 128, smem);
        if (e == cudaSuccess) {
            per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);   // 4 x 128 TMEM columns = the SM's 512
            // scene tiles on x, chunks of kMTiles model tiles on y: enough CTAs that two per SM overlap one
            // another's copies, products and epilogues even when the scene has few tiles
            constexpr int kMTiles = 8;
            const int64_t stiles = ((int64_t)S + TM - 1) / TM;
            const int mchunks = (R + TN * kMTiles - 1) / (TN * kMTiles);
            const int64_t gx = std::min<int64_t>(stiles, std::max<int64_t>(1, (int64_t)sms * per_sm * 8 / mchunks));
            unary_tma_kernel<<<dim3((unsigned)gx, (unsigned)mchunks), 128, smem, st>>>(
                tmA, tmB, S, R, Kp, snorm, mnorm, lambda1, U, ldu, TN * kMTiles, status);
            e = cudaGetLastError();
        }
    } else {
        e = launch_rowdot<kDist>(scene, S, ld, model, R, ld, F, snorm, mnorm, lambda1, nullptr, U, ldu, status, st);
    }
    prof_end(kProfUnary, st);
    return e;
}

cudaError_t launch_rowdot_plain(const float *X, int64_t nrows, int ldx, const float *W, int ncols, int ldw, int F,
                                const float *bias, float *Y, int64_t ldy, int *status, cudaStream_t st)
{
    return launch_rowdot<kPlain>(X, nrows, ldx, W, ncols, ldw, F, nullptr, nullptr, 0.0f, bias, Y, ldy, status, st);
}

}  // namespace hgm

// k_gemm_test.cu -- C = bf16(A) * bf16(B)^T with FP32 accumulation on the tensor cores
// (tcgen05.mma kind::f16, accumulator in tensor memory). A test hook that pins the
// operand layout and descriptors shared by the BF16 kernels of the library.
#include "hgm_internal.cuh"
#include "tc05.cuh"

namespace hgm {
namespace {

constexpr int TM = 128;          // rows per CTA (MMA M)
constexpr int TN = 128;          // columns per CTA (MMA N)
constexpr int KMAX = 256;        // K limit of this hook
constexpr uint32_t kLBO = 128;   // core matrices adjacent along K are contiguous
constexpr size_t kSlack = 16384;

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const float *__restrict__ A, const float *__restrict__ B, int M,
                                                        int N, int K, float *__restrict__ C, int *__restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // operand tiles, each followed by 16 KB of slack so that a descriptor read
    // with the two byte offsets exchanged still stays inside this CTA's shared memory
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    unsigned char *sA = smem;
    unsigned char *sB = smem + (size_t)TM * K * 2 + kSlack;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;

    if (warp == 0) tc05::tmem_alloc<TN>(&tslot);
    for (int e = tid; e < TM * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        const float v = (m0 + r < M) ? A[(int64_t)(m0 + r) * K + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16 *>(sA + tc05::kmajor_offset(r, k, kLBO, sbo)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < TN * K; e += blockDim.x) {
        const int r = e / K, k = e % K;
        const float v = (n0 + r < N) ? B[(int64_t)(n0 + r) * K + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16 *>(sB + tc05::kmajor_offset(r, k, kLBO, sbo)) = __float2bfloat16_rn(v);
    }
    if (tid == 0) tc05::mbar_init(&mbar, 1);
    tc05::fence_proxy_async_smem();
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t taddr = tslot;
    if (tid == 0) {
        const uint32_t a0 = tc05::smem_u32(sA), b0 = tc05::smem_u32(sB);
        constexpr uint32_t idesc = tc05::idesc_bf16_f32(TM, TN);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc05::smem_desc(a0 + ks * 2 * kLBO, kLBO, sbo);
            const uint64_t bd = tc05::smem_desc(b0 + ks * 2 * kLBO, kLBO, sbo);
            tc05::mma_bf16(taddr, ad, bd, idesc, ks > 0);
        }
        tc05::mma_commit(&mbar);
    }
    const bool ok = tc05::mbar_wait(&mbar, 0, 1u << 26);
    if (!ok && lane == 0) atomicExch(status, 1);
    tc05::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < TN; c0 += 32) {
            float v[32];
            tc05::tmem_ld32(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            const int row = m0 + 32 * warp + lane;
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (n0 + c0 + j < N) C[(int64_t)row * N + n0 + c0 + j] = v[j];
            }
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc<TN>(taddr);
}

}  // namespace
}  // namespace hgm

extern "C" hgm_status hgm_gemm_bf16(const float *A, const float *B, int32_t M, int32_t N, int32_t K, void *stream,
                                    float *C, int32_t *status)
{
    if (M < 1 || N < 1 || K < 16 || K > hgm::KMAX || K % 16 != 0 || !A || !B || !C || !status)
        return hgm::set_error(HGM_EINVAL, "hgm_gemm_bf16: M, N >= 1, K a multiple of 16 in 16..256");
    const size_t smem = (size_t)hgm::TM * K * 2 + (size_t)hgm::TN * K * 2 + 2 * hgm::kSlack;
    cudaError_t e = cudaFuncSetAttribute(hgm::gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return hgm::set_error(HGM_ECUDA, cudaGetErrorString(e));
    dim3 grid((unsigned)((M + hgm::TM - 1) / hgm::TM), (unsigned)((N + hgm::TN - 1) / hgm::TN));
    hgm::gemm_bf16_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(A, B, M, N, K, C, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return hgm::set_error(HGM_ECUDA, cudaGetErrorString(e));
    return HGM_OK;
}

// k_debug.cu -- test hooks for device helpers that have no entry point of their own.
#include "fast_math.cuh"
#include "hgm_internal.cuh"
#include "tc05.cuh"

namespace hgm {
namespace {

__global__ void atan2_kernel(const float *__restrict__ y, const float *__restrict__ x, int64_t n,
                             float *__restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = fast_atan2(y[k], x[k]);
}

// A bounded wait that runs out: an mbarrier that nothing arrives on, waited on with the same helper the
// tensor-core kernels use; the kernel records the timeout in *status and returns.
__global__ void timeout_kernel(uint32_t polls, int32_t *status)
{
    __shared__ uint64_t mbar;
    if (threadIdx.x == 0) tc05::mbar_init(&mbar, 1);
    __syncthreads();
    const bool ok = tc05::mbar_wait(&mbar, 0, polls);
    if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) *status = 1;
}

}  // namespace
}  // namespace hgm

extern "C" hgm_status hgm_debug_timeout(uint32_t polls, void *stream, int32_t *status)
{
    if (!status || polls == 0 || polls > (1u << 20)) return hgm::set_error(HGM_EINVAL, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) {
        hgm::timeout_kernel<<<1, 32, 0, st>>>(polls, status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return hgm::set_error(HGM_ECUDA, cudaGetErrorString(e));
    return HGM_OK;
}

extern "C" hgm_status hgm_atan2_f32(const float *y, const float *x, int64_t n, void *stream, float *out)
{
    if (n < 0 || (n > 0 && (!y || !x || !out))) return hgm::set_error(HGM_EINVAL, "bad arguments");
    if (n == 0) return HGM_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    hgm::atan2_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(y, x, n, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return hgm::set_error(HGM_ECUDA, cudaGetErrorString(e));
    return HGM_OK;
}

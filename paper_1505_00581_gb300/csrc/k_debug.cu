// k_debug.cu -- test hooks for device helpers that have no entry point of their own.
#include "fast_math.cuh"
#include "hgm_internal.cuh"

namespace hgm {
namespace {

__global__ void atan2_kernel(const float *__restrict__ y, const float *__restrict__ x, int64_t n,
                             float *__restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = fast_atan2(y[k], x[k]);
}

}  // namespace
}  // namespace hgm

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

// unary_common.cuh -- the FP32 unary cost of one (model point, scene point) pair with the rounding of the
// FP32 unary table (Eq. 2): d_k = f_k - f'_k, s = fma(d_k, d_k, s) for k in order, IEEE sqrt, times lambda1.
// Used wherever the precision mode re-scores candidates, so that a re-scored cost equals the table's.
#pragma once

namespace hgm {

__device__ __forceinline__ float unary_fp32(const float *a, const float *b, int F, float lambda1)
{
    float s = 0.0f;
    if ((F & 3) == 0) {   // rows padded to a multiple of 4 floats and 16-byte aligned: same order, float4 reads
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const float4 *b4 = reinterpret_cast<const float4 *>(b);
        for (int k = 0; k < (F >> 2); ++k) {
            const float4 x = a4[k], y = b4[k];
            float d = __fsub_rn(x.x, y.x);
            s = __fmaf_rn(d, d, s);
            d = __fsub_rn(x.y, y.y);
            s = __fmaf_rn(d, d, s);
            d = __fsub_rn(x.z, y.z);
            s = __fmaf_rn(d, d, s);
            d = __fsub_rn(x.w, y.w);
            s = __fmaf_rn(d, d, s);
        }
    } else if ((F & 1) == 0 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 7) == 0) {
        // even F with 8-byte aligned rows (F = 162): the same order, float2 reads
        const float2 *a2 = reinterpret_cast<const float2 *>(a);
        const float2 *b2 = reinterpret_cast<const float2 *>(b);
        for (int k = 0; k < (F >> 1); ++k) {
            const float2 x = a2[k], y = b2[k];
            float d = __fsub_rn(x.x, y.x);
            s = __fmaf_rn(d, d, s);
            d = __fsub_rn(x.y, y.y);
            s = __fmaf_rn(d, d, s);
        }
    } else {
        for (int k = 0; k < F; ++k) {
            const float d = __fsub_rn(a[k], b[k]);
            s = __fmaf_rn(d, d, s);
        }
    }
    return __fmul_rn(lambda1, __fsqrt_rn(s));
}

}  // namespace hgm

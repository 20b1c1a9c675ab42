// recurse_common.cuh -- the per-triple arithmetic shared by both recursion kernels.
//
// Each helper fixes the FP32 operations and their rounding explicitly (no
// compiler contraction choices), so the large-list and the short-list kernels
// produce the same bits for the same inputs.
#pragma once

#include "f32x2.cuh"
#include "fast_math.cuh"
#include "hgm_internal.cuh"

namespace hgm {

__device__ __forceinline__ float sqrt_fast(float x)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// one fold of an angle in [-3pi, 3pi] to [-pi, pi]
__device__ __forceinline__ float wrap_pi(float v)
{
    if (v > kPi) v = __fsub_rn(v, kTwoPi);
    else if (v < -kPi) v = __fadd_rn(v, kTwoPi);
    return v;
}

// signed angle at v from v->p to v->q (reading R1)
__device__ __forceinline__ float signed_angle(float2 v, float2 p, float2 q)
{
    return wrap_pi(__fsub_rn(fast_atan2(__fsub_rn(q.y, v.y), __fsub_rn(q.x, v.x)),
                             fast_atan2(__fsub_rn(p.y, v.y), __fsub_rn(p.x, v.x))));
}

// theta(p->q)
__device__ __forceinline__ float direction(float2 p, float2 q)
{
    return fast_atan2(__fsub_rn(q.y, p.y), __fsub_rn(q.x, p.x));
}

// base(a,b) = U(a) + lambda2 |dt_model - (t'(a) - t'(b))| + alpha_{i+1}(a,b)
__device__ __forceinline__ float base_cost(float u, float lam2, int dt_model, int ta, int tb, float alpha)
{
    return __fadd_rn(__fmaf_rn(lam2, fabsf((float)(dt_model - (ta - tb))), u), alpha);
}

// v(a,b,c) = base + lambda2 lambda3 sqrt(d1^2 + d2^2), d1 = p1 - q1, d2 = p1 + k2 - r (circular folds)
__device__ __forceinline__ float triple_cost(float base, float p1, float p2, float q1, float r, float lam23)
{
    const float d1 = __fsub_rn(p1, q1);
    const float d2 = __fsub_rn(p2, r);
    const float w1 = fminf(fabsf(d1), __fsub_rn(kTwoPi, fabsf(d1)));
    const float w2 = fminf(fabsf(d2), __fsub_rn(kTwoPi, fabsf(d2)));
    return __fmaf_rn(lam23, sqrt_fast(__fmaf_rn(w2, w2, __fmul_rn(w1, w1))), base);
}

// triple_cost for two cells (same a, b; c and c'): bit-identical to two triple_cost calls.
// p1p = (p1, p1), p2p = (p2, p2), basep = (base, base), lam = (lambda2 lambda3, lambda2 lambda3).
__device__ __forceinline__ void triple_cost2(unsigned long long basep, unsigned long long p1p,
                                             unsigned long long p2p, unsigned long long q1p, unsigned long long rp,
                                             unsigned long long lam, float &va, float &vb)
{
    float d1a, d1b, d2a, d2b;
    upk2(sub2(p1p, q1p), d1a, d1b);
    upk2(sub2(p2p, rp), d2a, d2b);
    const float w1a = fminf(fabsf(d1a), __fsub_rn(kTwoPi, fabsf(d1a)));
    const float w1b = fminf(fabsf(d1b), __fsub_rn(kTwoPi, fabsf(d1b)));
    const float w2a = fminf(fabsf(d2a), __fsub_rn(kTwoPi, fabsf(d2a)));
    const float w2b = fminf(fabsf(d2b), __fsub_rn(kTwoPi, fabsf(d2b)));
    const unsigned long long w1 = pk2(w1a, w1b), w2 = pk2(w2a, w2b);
    float sa, sb;
    upk2(fma2(w2, w2, mul2(w1, w1)), sa, sb);
    upk2(fma2(lam, pk2(sqrt_fast(sa), sqrt_fast(sb)), basep), va, vb);
}

// alpha_i(b,c) = min_a v + lambda2 |dt_model - (t'(b) - t'(c))|
__device__ __forceinline__ float cell_alpha(float best, float lam2, int dt_model, int tb, int tc)
{
    return __fmaf_rn(lam2, fabsf((float)(dt_model - (tb - tc))), best);
}

}  // namespace hgm

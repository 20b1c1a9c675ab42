// fast_math.cuh -- FP32 two-argument arctangent for the recursion kernel.
//
// atan2(y, x) by octant reduction to r = min(|x|,|y|) / max(|x|,|y|) in [0, 1]
// and atan(r) ~= r * P(r^2), P of degree 6 fitted by weighted least squares
// with Lawson reweighting towards the minimax error (`python csrc/fit_atan.py`,
// default degree 6, prints these coefficients and "max |err| = 2.474e-07 rad",
// the fit's FP64 error; the FP32 evaluation adds a few 1e-8). Then atan = pi/2 - a above the diagonal, pi - a for a
// negative (sign bit set) x, and the sign of y. atan2(0, 0) = 0.
#pragma once

namespace hgm {

__device__ __forceinline__ float fast_atan2(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float r = mx > 0.0f ? __fdividef(mn, mx) : 0.0f;
    const float s = r * r;
    float p = 6.811788903e-03f;
    p = fmaf(p, s, -3.360421455e-02f);
    p = fmaf(p, s, 7.962367824e-02f);
    p = fmaf(p, s, -1.323334354e-01f);
    p = fmaf(p, s, 1.980781645e-01f);
    p = fmaf(p, s, -3.331736826e-01f);
    p = fmaf(p, s, 9.999961117e-01f);
    float a = r * p;
    if (ay > ax) a = 1.57079632679489662f - a;
    if (signbit(x)) a = 3.14159265358979324f - a;
    return copysignf(a, y);
}

}  // namespace hgm

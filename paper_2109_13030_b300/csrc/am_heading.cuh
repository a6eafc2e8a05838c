// Heading helpers shared by the fused kernels: the atan2 of the heading
// target (Sec. III-D, heading step) and the wrap of an angle difference.
#pragma once

namespace trajam {
namespace {

constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kPi = 3.14159265358979323846f;

// atan2 for the heading target psi_t = atan2(s, c).  Octant reduction to
// a = min(|x|, |y|) / max(|x|, |y|) in [0, 1], atan(a) = a P(a^2) with P of
// degree 8 fitted for this kernel (iteratively reweighted least squares,
// Lawson's method, on [0, 1]: relative error 1.5e-8 in exact arithmetic,
// within 2 ulp when evaluated in FP32), then the octant is restored.
// atan2(0, 0) = 0, the reading the method takes.
__device__ __constant__ const float kAtanPoly[9] = {1.0f, -0.33333072f, 0.1999262f, -0.14203647f, 0.106409416f,
                                                    -0.07504311f, 0.042691723f, -0.016068758f, 0.002849923f};

__device__ __forceinline__ float atan2_heading(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float a = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float s = a * a;
    float p = kAtanPoly[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) p = fmaf(p, s, kAtanPoly[k]);
    float r = a * p;
    if (ay > ax) r = 1.57079637f - r;
    if (x < 0.f) r = 3.14159274f - r;
    return copysignf(r, y);  // the sign of y, -0 included (atan2(-0, -1) = -pi)
}

// Wrap into (-pi, pi].
__device__ __forceinline__ float wrap_pi(float a)
{
    return a - kTwoPi * ceilf((a - kPi) * (1.0f / kTwoPi));
}

}  // namespace
}  // namespace trajam

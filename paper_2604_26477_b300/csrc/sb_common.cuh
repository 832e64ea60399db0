// Device helpers shared by the single-instance and batched SB samplers.
#pragma once

#include "moq_common.cuh"

namespace moq {

// phi(x): sgn(x) with sgn(0) = +1 for dSB (x is never -0 in the samplers: the start state
// is sanitised and the update cannot produce -0 from +-nonzero or +0), x for bSB.
template <int VARIANT>
__device__ __forceinline__ float phi_of(float x)
{
    if (VARIANT == MOQ_DSB) return __int_as_float(0x3f800000 | (__float_as_int(x) & 0x80000000));
    return x;
}

// Symplectic Euler update of one spin given its force f (SB equations, Eq. NI-SB):
// y += dt (-(a0 - a_m) x + f) + kappa eta; x += dt a0 y; inelastic wall at |x| > 1.
template <bool NOISE>
__device__ __forceinline__ void sb_update(float f, float cm, float eta, float dt, float kappa, float dta0, float& x, float& y)
{
    const float drift = fmaf(cm, x, f);
    y = fmaf(dt, drift, y);
    if (NOISE) y = fmaf(kappa, eta, y);
    x = fmaf(dta0, y, x);
    if (fabsf(x) > 1.0f) {
        x = copysignf(1.0f, x);
        y = 0.0f;
    }
}

// The same update for the two replicas of a pair at once: every multiply-add is one
// packed two-lane FP32 instruction (each lane rounds as the scalar fmaf does, so both forms
// give the same bits); the wall is applied per lane.
template <bool NOISE>
__device__ __forceinline__ void sb_update2(float2 f, float2 cm, float2 eta, float2 dt, float2 kappa, float2 dta0, float2& x, float2& y)
{
    const float2 drift = __ffma2_rn(cm, x, f);
    y = __ffma2_rn(dt, drift, y);
    if (NOISE) y = __ffma2_rn(kappa, eta, y);
    x = __ffma2_rn(dta0, y, x);
    if (fabsf(x.x) > 1.0f) {
        x.x = copysignf(1.0f, x.x);
        y.x = 0.0f;
    }
    if (fabsf(x.y) > 1.0f) {
        x.y = copysignf(1.0f, x.y);
        y.y = 0.0f;
    }
}

}  // namespace moq

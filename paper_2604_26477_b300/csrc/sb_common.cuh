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

}  // namespace moq

// gsb_update.cuh -- the per-oscillator part of one time step (Sec. II).
#pragma once
#include "gsb_internal.cuh"

namespace gsb {

__device__ __forceinline__ float sgnf(float v) { return v >= 0.f ? 1.f : -1.f; }

// One oscillator, given the coupling f = (J v)_i at t_m:
//   FP  (Eq. 7): p <- p - (1 - A x^2) p / (M - m)   (individual control), or the
//                shared p(t_{m+1}) (Eq. 6 / caller schedule)
//   FX  (Eq. 3): y <- y - (p x - c f) dt, with p(t_{m+1}) and x(t_m)
//   FY  (Eq. 4): x <- x + y dt
//   wall (Eq. 5): |x| > 1 -> x = sgn x, y = 0
// inv_rem = 1 / (M - m) rounded to FP32 (a multiply replaces the divide).
template <bool CONTROL>
__device__ __forceinline__ void sb_update(float& x, float& y, float& p, float f, float a,
                                          float c, float dt, float p_shared, float inv_rem) {
    const float xo = x;
    float pn;
    if (CONTROL)
        pn = p - (1.f - a * xo * xo) * p * inv_rem;
    else
        pn = p_shared;
    float yn = y - (pn * xo - c * f) * dt;
    float xn = xo + yn * dt;
    if (fabsf(xn) > 1.f) {
        xn = sgnf(xn);
        yn = 0.f;
    }
    x = xn;
    y = yn;
    p = pn;
}

}  // namespace gsb

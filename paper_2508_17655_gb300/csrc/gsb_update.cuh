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
// Every operation is an explicit round-to-nearest multiply or fused
// multiply-add in a fixed order, with the negations folded into the constants
// (exact), so sb_update2 below -- the same sequence on two oscillators per
// instruction -- gives identical bits, and no compiler contraction choice
// differs between kernels.
template <bool CONTROL>
__device__ __forceinline__ void sb_update(float& x, float& y, float& p, float f, float a,
                                          float c, float dt, float p_shared, float inv_rem) {
    const float xo = x;
    float pn;
    if (CONTROL) {
        const float t = __fmul_rn(-a, xo);           // -A x
        const float g = __fmaf_rn(t, xo, 1.f);       // 1 - A x^2
        const float q = __fmul_rn(g, p);             // (1 - A x^2) p
        pn = __fmaf_rn(q, -inv_rem, p);              // p - (1 - A x^2) p / (M - m)
    } else {
        pn = p_shared;
    }
    const float ncf = __fmul_rn(-c, f);              // -c f
    const float u = __fmaf_rn(pn, xo, ncf);          // p x - c f
    float yn = __fmaf_rn(u, -dt, y);                 // y - (p x - c f) dt
    float xn = __fmaf_rn(yn, dt, xo);                // x + y dt
    if (fabsf(xn) > 1.f) {
        xn = sgnf(xn);
        yn = 0.f;
    }
    x = xn;
    y = yn;
    p = pn;
}

// sb_update on two oscillators at once (packed FP32 pairs, sm_100 and later):
// the same operations in the same order, each element rounded as above.
template <bool CONTROL>
__device__ __forceinline__ void sb_update2(float2& x, float2& y, float2& p, float2 f, float a,
                                           float c, float dt, float p_shared, float inv_rem) {
    const float2 xo = x;
    float2 pn;
    if (CONTROL) {
        const float2 t = __fmul2_rn(make_float2(-a, -a), xo);
        const float2 g = __ffma2_rn(t, xo, make_float2(1.f, 1.f));
        const float2 q = __fmul2_rn(g, p);
        pn = __ffma2_rn(q, make_float2(-inv_rem, -inv_rem), p);
    } else {
        pn = make_float2(p_shared, p_shared);
    }
    const float2 ncf = __fmul2_rn(make_float2(-c, -c), f);
    const float2 u = __ffma2_rn(pn, xo, ncf);
    float2 yn = __ffma2_rn(u, make_float2(-dt, -dt), y);
    float2 xn = __ffma2_rn(yn, make_float2(dt, dt), xo);
    if (fabsf(xn.x) > 1.f) {
        xn.x = sgnf(xn.x);
        yn.x = 0.f;
    }
    if (fabsf(xn.y) > 1.f) {
        xn.y = sgnf(xn.y);
        yn.y = 0.f;
    }
    x = xn;
    y = yn;
    p = pn;
}

}  // namespace gsb

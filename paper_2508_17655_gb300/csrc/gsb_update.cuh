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

// Tangent-linear form of sb_update (the step linearised in (x, y, p)):
//   dp' = dp - [(1 - A x^2) dp - 2 A x dx p] / (M - m)   (individual control; 0 otherwise)
//   dy' = dy - [dp' x + p' dx - c df] dt                 (df = (J dx)_i; none for sgn coupling)
//   dx' = dx + dy' dt;  where Eq. 5 clamps x', also dx' = dy' = 0.
template <bool CONTROL, bool SIGN>
__device__ __forceinline__ void sb_tangent_update(float& x, float& y, float& p, float& dx,
                                                  float& dy, float& dp, float f, float df,
                                                  float a, float c, float dt, float p_shared,
                                                  float inv_rem) {
    const float xo = x, dxo = dx;
    float pn, dpn;
    if (CONTROL) {
        const float g = 1.f - a * xo * xo;
        dpn = dp - (g * dp - 2.f * a * xo * dxo * p) * inv_rem;
        pn = p - g * p * inv_rem;
    } else {
        pn = p_shared;
        dpn = 0.f;
    }
    const float dfi = SIGN ? 0.f : df;
    float dyn = dy - (dpn * xo + pn * dxo - c * dfi) * dt;
    float yn = y - (pn * xo - c * f) * dt;
    float xn = xo + yn * dt;
    float dxn = dxo + dyn * dt;
    if (fabsf(xn) > 1.f) {
        xn = sgnf(xn);
        yn = 0.f;
        dxn = 0.f;
        dyn = 0.f;
    }
    x = xn;
    y = yn;
    p = pn;
    dx = dxn;
    dy = dyn;
    dp = dpn;
}

// bf16 bits of a finite v rounded to nearest even, by integer operations (no
// conversion instruction): add just under half a bf16 ulp (0x7FFF), plus one
// when the kept part is odd so that ties go to the even neighbour, and keep
// the top 16 bits. A carry out of the mantissa moves into the exponent, as the
// rounding requires.
__device__ __forceinline__ uint32_t bf16_rne_bits(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
}
// x = x_hi + x_lo with x_hi = bf16(x) and x_lo = bf16(x - x_hi) (x - x_hi is
// exact in FP32: the two agree in their top 8 bits); both as bf16 bits.
__device__ __forceinline__ void bf16_split_bits(float v, uint32_t& hi, uint32_t& lo) {
    hi = bf16_rne_bits(v);
    lo = bf16_rne_bits(v - __uint_as_float(hi << 16));
}

}  // namespace gsb

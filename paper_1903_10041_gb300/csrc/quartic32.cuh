// Quartic minimiser for the mixed-precision solver: Algorithm 1 (Sec. III-B)
// evaluated in FP32, with every branch decision of the cubic taken as FP64
// would take it.
//
// Same mathematics as quartic64.cuh.  Differences:
//  * The sign of Delta = Q^3 + R^2 is computed in FP32 together with a
//    forward error bound (first-order propagation of one unit roundoff per
//    FP32 operation through b, c, d, Q, R and Delta, with a safety factor
//    of at least 1.25 on every term).  When |Delta| exceeds the bound the
//    FP32 sign is the exact sign, and therefore FP64's.  Otherwise b, c, d, Q, R
//    and Delta are recomputed in FP64 from the same A, B, C, D and the FP64
//    values decide the branch (and the Q = R = 0 test).
//  * The closed-form roots lose about log10(|b|/|x|) digits to cancellation
//    in FP32, so each candidate gets one Newton step on the derivative of
//    the original quartic, 4A x^3 + 3B x^2 + 2C x + D, which is evaluated
//    without that cancellation.  The step is taken
//    only where the quartic is convex (a minimiser) and the step is small,
//    so it cannot jump to another root.
//  * The two minima are compared through the factored difference
//    F(u) - F(v) = (u - v) [ (u^3 + u^2 v + u v^2 + v^3)/4 + (b/3)(u^2 + u v + v^2)
//                            + (c/2)(u + v) + d ],
//    which is the delta-f of Algorithm 1 without its cancellation.
#pragma once
#include "common.cuh"
#include "quartic64.cuh"

namespace admm_impl {

// Fast FP32 primitives for the closed forms.  Their few-ulp errors are
// removed by the Newton step that follows (the root it converges to depends
// only on the coefficients), and the discriminant bound below allows for a
// reciprocal that is off by 2 ulp.
__device__ __forceinline__ float rcp_fast(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ float sqrt_fast(float v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }
__device__ __forceinline__ float cbrt_fast(float v)
{
    const float a = fabsf(v);
    const float r = a > 0.0f ? exp2f(__log2f(a) * (1.0f / 3.0f)) : 0.0f;
    return copysignf(r, v);
}

// The FP64 closed form, out of line: taken only when FP32 overflows.
static __device__ __noinline__ float quartic_min_fallback64(float A, float B, float C, float D, float lo, float hi,
                                                     int paper_mode)
{
    return (float)quartic_min64((double)A, (double)B, (double)C, (double)D, (double)lo, (double)hi, paper_mode);
}

// One Horner step s <- s x + a with its rounding errors carried in c
// (compensated Horner scheme: error-free product by FMA, TwoSum for the
// addition; Graillat, Langlois and Louvet, 2005).
__device__ __forceinline__ void horner_comp_step(float &s, float &c, float x, float a)
{
    const float p = __fmul_rn(s, x);
    const float pe = __fmaf_rn(s, x, -p);
    const float t = __fadd_rn(p, a);
    const float bb = __fsub_rn(t, p);
    const float se = __fadd_rn(__fsub_rn(p, __fsub_rn(t, bb)), __fsub_rn(a, bb));
    s = t;
    c = __fmaf_rn(c, x, __fadd_rn(pe, se));
}

// Newton step on the quartic's derivative 4A x^3 + 3B x^2 + 2C x + D in
// FP32 Horner form.  Built with ADMM_COMPENSATED_POLISH, the derivative is
// evaluated by the compensated Horner scheme instead (about twice the
// working precision: the polished root is then the FP32 number nearest the
// root of the FP32 coefficients rather than up to a few units off it).
__device__ __forceinline__ float newton_polish32(float A, float B, float C, float D, float x)
{
#ifndef ADMM_COMPENSATED_POLISH
    const float fp = ((4.0f * A * x + 3.0f * B) * x + 2.0f * C) * x + D;
#else
    float s = 4.0f * A, c = 0.0f;
    horner_comp_step(s, c, x, 3.0f * B);
    horner_comp_step(s, c, x, 2.0f * C);
    horner_comp_step(s, c, x, D);
    const float fp = s + c;
#endif
    const float fpp = (12.0f * A * x + 6.0f * B) * x + 2.0f * C;
    if (fpp > 0.0f) {
        const float dx = fp * rcp_fast(fpp);
        if (fabsf(dx) <= 0.0625f * (fabsf(x) + 1.0f)) x -= dx;
    }
    return x;
}

// Sign of F(u) - F(v) via the factored form (F' = x^3 + b x^2 + c x + d).
__device__ __forceinline__ float delta_f32(float u, float v, float b, float c, float d)
{
    const float br = 0.25f * (u * u * u + u * u * v + u * v * v + v * v * v) +
                     (b * (1.0f / 3.0f)) * (u * u + u * v + v * v) + 0.5f * c * (u + v) + d;
    return (u - v) * br;
}

// FP64-cubic variant: b, c, d, Q, R, Delta, roots and delta-f in FP64.
__device__ __forceinline__ float quartic_min_fp64cubic(float A, float B, float C, float D, float lo, float hi,
                                                       int paper_mode)
{
    return (float)quartic_min64((double)A, (double)B, (double)C, (double)D, (double)lo, (double)hi, paper_mode);
}

// The branch of Algorithm 1 decided in FP64 from the same A, B, C, D.
static __device__ __noinline__ int cubic_branch64(float A, float B, float C, float D)
{
    const double inv64 = 1.0 / (double)A;
    const double bd = 0.75 * (double)B * inv64, cd = 0.5 * (double)C * inv64, dd = 0.25 * (double)D * inv64;
    const double b3d = bd * (1.0 / 3.0);
    const double Qd = cd * (1.0 / 3.0) - b3d * b3d;
    const double Rd = b3d * (0.5 * cd) - b3d * b3d * b3d - 0.5 * dd;
    const double Dd = Qd * Qd * Qd + Rd * Rd;
    return Dd > 0.0 ? 0 : ((Qd == 0.0 && Rd == 0.0) ? 1 : 2);
}

// FP32 variant with FP64-certified branch decisions.  `esc` counts the
// decisions that needed FP64.
__device__ __forceinline__ float quartic_min32(float A, float B, float C, float D, float lo, float hi,
                                               int paper_mode, unsigned &esc)
{
    if (A == 0.0f) return clampf(-D * rcp_fast(2.0f * C), lo, hi);
    const float inv = rcp_fast(A);
    const float b = 0.75f * B * inv, c = 0.5f * C * inv, d = 0.25f * D * inv;
    const float b3 = b * (1.0f / 3.0f);
    const float Q = c * (1.0f / 3.0f) - b3 * b3;
    const float R = b3 * (0.5f * c) - b3 * b3 * b3 - 0.5f * d;
    const float Q3 = Q * Q * Q, R2 = R * R;
    const float Dl = Q3 + R2;
    // magnitudes entering Q, R (including the rounding of b, c, d)
    const float mQ = fabsf(c) * (1.0f / 3.0f) + b3 * b3;
    const float mR = fabsf(b3 * 0.5f * c) + fabsf(b3 * b3 * b3) + 0.5f * fabsf(d);
    // |fl(Delta) - Delta| <= u (78 Q^2 mQ + 12 |Q|^3 + 88 |R| mR + 4 R^2) with u = 2^-24
    // (a factor 2 over the first-order propagation of the roundings above,
    // with a reciprocal of A off by up to 2 ulp); the constants below
    // dominate each term.
    const float bound = 6.0e-8f * (96.0f * Q * Q * mQ + 64.0f * fabsf(Q3) + 96.0f * fabsf(R) * mR + 64.0f * R2);
    int branch; // 0 Cardano, 1 triple, 2 trig
    if (Dl > bound) branch = 0;
    else if (Dl < -bound) branch = 2;
    else {
        ++esc;
        branch = cubic_branch64(A, B, C, D);
    }
    if (branch == 1) return clampf(-b3, lo, hi);
    if (branch == 0) {
        const float sq = sqrt_fast(Dl);
        const float S = cbrt_fast(R >= 0.0f ? R + sq : R - sq);
        const float T = S != 0.0f ? -Q * rcp_fast(S) : 0.0f;
        const float x = newton_polish32(A, B, C, D, S + T - b3);
        if (!isfinite(x)) return quartic_min_fallback64(A, B, C, D, lo, hi, paper_mode);
        return clampf(x, lo, hi);
    }
    // three real roots: t = theta/3 lies in [0, pi/3], where the fast sine and
    // cosine are accurate to a few ulp; the Newton step below removes their error
    const float nQ = fmaxf(-Q, 0.0f);
    const float arg = nQ > 0.0f ? fminf(fmaxf(R * rsqrtf(nQ * nQ * nQ), -1.0f), 1.0f) : (R >= 0.0f ? 1.0f : -1.0f);
    const float t = acosf(arg) * (1.0f / 3.0f);
    const float st = __sinf(t), ct = __cosf(t);
    const float two_sq = 2.0f * sqrt_fast(nQ);
    float x3 = two_sq * ct - b3;
    float x1 = two_sq * (-0.5f * ct - 0.86602540378f * st) - b3;
    x1 = newton_polish32(A, B, C, D, x1);
    x3 = newton_polish32(A, B, C, D, x3);
    if (!isfinite(x1) || !isfinite(x3)) return quartic_min_fallback64(A, B, C, D, lo, hi, paper_mode);
    if (paper_mode) {
        const float xs = delta_f32(x1, x3, b, c, d) > 0.0f ? x3 : x1;
        return clampf(xs, lo, hi);
    }
    const float u = clampf(x1, lo, hi), v = clampf(x3, lo, hi);
    return delta_f32(u, v, b, c, d) > 0.0f ? v : u;
}

} // namespace admm_impl

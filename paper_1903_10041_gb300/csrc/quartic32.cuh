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
    // the operations and roundings of newton_polish32x2, lane for lane
    const float C2 = __fadd_rn(C, C);
    const float fp = __fmaf_rn(__fmaf_rn(__fmaf_rn(__fmul_rn(4.0f, A), x, __fmul_rn(3.0f, B)), x, C2), x, D);
    const float fpp = __fmaf_rn(__fmaf_rn(__fmul_rn(12.0f, A), x, __fmul_rn(6.0f, B)), x, C2);
    if (fpp > 0.0f) {
        const float dx = __fmul_rn(fp, rcp_fast(fpp));
        if (fabsf(dx) <= __fmul_rn(0.0625f, __fadd_rn(fabsf(x), 1.0f))) x = __fsub_rn(x, dx);
    }
    return x;
#else
    float s = 4.0f * A, c = 0.0f;
    horner_comp_step(s, c, x, 3.0f * B);
    horner_comp_step(s, c, x, 2.0f * C);
    horner_comp_step(s, c, x, D);
    const float fp = s + c;
    const float fpp = (12.0f * A * x + 6.0f * B) * x + 2.0f * C;
    if (fpp > 0.0f) {
        const float dx = fp * rcp_fast(fpp);
        if (fabsf(dx) <= 0.0625f * (fabsf(x) + 1.0f)) x -= dx;
    }
    return x;
#endif
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
    // Every operation below is rounded as the packed path (quartic_min32x2)
    // rounds it, so a lane gets the same bits on either path.
    if (A == 0.0f) return clampf(__fmul_rn(-D, rcp_fast(__fadd_rn(C, C))), lo, hi);
    const float inv = rcp_fast(A);
    const float b = __fmul_rn(__fmul_rn(0.75f, B), inv);
    const float c = __fmul_rn(__fmul_rn(0.5f, C), inv);
    const float d = __fmul_rn(__fmul_rn(0.25f, D), inv);
    const float b3 = __fmul_rn(b, 1.0f / 3.0f);
    const float b3s = __fmul_rn(b3, b3), b3c = __fmul_rn(b3s, b3);
    const float Q = __fmaf_rn(c, 1.0f / 3.0f, -b3s);
    const float bhc = __fmul_rn(b3, __fmul_rn(0.5f, c));
    const float R = __fsub_rn(__fsub_rn(bhc, b3c), __fmul_rn(0.5f, d));
    const float Qs = __fmul_rn(Q, Q);
    const float Dl = __fadd_rn(__fmul_rn(Qs, Q), __fmul_rn(R, R));
    // magnitudes entering Q, R (including the rounding of b, c, d); |Q| <= mQ and |R| <= mR
    const float mQ = __fmaf_rn(fabsf(c), 1.0f / 3.0f, b3s);
    const float mR = __fmaf_rn(0.5f, fabsf(d), __fadd_rn(fabsf(bhc), fabsf(b3c)));
    // |fl(Delta) - Delta| <= u (78 Q^2 mQ + 12 |Q|^3 + 88 |R| mR + 4 R^2) with u = 2^-24
    // (a factor 2 over the first-order propagation of the roundings above,
    // with a reciprocal of A off by up to 2 ulp).  As |Q|^3 <= Q^2 mQ and
    // R^2 <= |R| mR, that is at most 92 u (Q^2 mQ + |R| mR); the bound takes
    // 128 u (Q^2 mQ + |R| mR), a safety factor of 1.39.
    const float bound = __fmul_rn(7.68e-6f, __fmaf_rn(Qs, mQ, __fmul_rn(fabsf(R), mR)));
    int branch; // 0 Cardano, 1 triple, 2 trig
    if (Dl > bound) branch = 0;
    else if (Dl < -bound) branch = 2;
    else {
        ++esc;
        branch = cubic_branch64(A, B, C, D);
    }
    if (branch == 1) return clampf(-b3, lo, hi);
    if (branch == 0) {
        // Delta > 0 here (certified, or FP64 said so): as in the packed path
        const float sq = Dl > 0.0f ? __fmul_rn(Dl, rsqrtf(Dl)) : 0.0f;
        const float S = cbrt_fast(__fadd_rn(R, R >= 0.0f ? sq : -sq));
        const float T = S != 0.0f ? __fmul_rn(-Q, rcp_fast(S)) : 0.0f;
        const float x = newton_polish32(A, B, C, D, __fsub_rn(__fadd_rn(S, T), b3));
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

// ---------------------------------------------------------------------------
// FP64 minimiser seeded in FP32.  FP64 throughput is 1/64 of FP32 on this
// GPU, so for the Cardano branch the root is found in FP32 (closed form +
// Newton step, as in quartic_min32) and then refined by two FP64 Newton steps
// on the FP64 derivative 4A x^3 + 3B x^2 + 2C x + D (step divisor from an
// FP32 reciprocal: each step multiplies the relative error by about the
// FP32 unit roundoff, so two steps reach FP64 rounding).  The FP32 branch
// test is certified against the FP64 coefficients: the error bound of
// quartic_min32 is doubled for the rounding of A, B, C, D to FP32.  Anything
// else (quadratic, trig or uncertain branch, FP32 range, a step that did not
// settle) takes the FP64 closed form of quartic_min64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool cardano_seed32(double A64, double B64, double C64, double D64, float &root)
{
    const float A = (float)A64, B = (float)B64, C = (float)C64, D = (float)D64;
    if (!(A > 1.0e-30f && A < 1.0e30f)) return false;
    const float inv = rcp_fast(A);
    const float b = 0.75f * B * inv, c = 0.5f * C * inv, d = 0.25f * D * inv;
    const float b3 = b * (1.0f / 3.0f);
    const float Q = c * (1.0f / 3.0f) - b3 * b3;
    const float R = b3 * (0.5f * c) - b3 * b3 * b3 - 0.5f * d;
    const float Q3 = Q * Q * Q, R2 = R * R;
    const float Dl = Q3 + R2;
    const float mQ = fabsf(c) * (1.0f / 3.0f) + b3 * b3;
    const float mR = fabsf(b3 * 0.5f * c) + fabsf(b3 * b3 * b3) + 0.5f * fabsf(d);
    const float bound = 1.2e-7f * (96.0f * Q * Q * mQ + 64.0f * fabsf(Q3) + 96.0f * fabsf(R) * mR + 64.0f * R2);
    if (!(Dl > bound)) return false;
    const float sq = sqrt_fast(Dl);
    const float S = cbrt_fast(R >= 0.0f ? R + sq : R - sq);
    const float T = S != 0.0f ? -Q * rcp_fast(S) : 0.0f;
    root = newton_polish32(A, B, C, D, S + T - b3);
    return isfinite(root);
}

__device__ __forceinline__ double quartic_min64_seeded(double A, double B, double C, double D, double lo, double hi,
                                                       int paper_mode)
{
    float r32;
    if (A != 0.0 && cardano_seed32(A, B, C, D, r32)) {
        const double A4 = 4.0 * A, B3 = 3.0 * B, C2 = 2.0 * C, A12 = 12.0 * A, B6 = 6.0 * B;
        double x = (double)r32, step = 0.0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const double p = ((A4 * x + B3) * x + C2) * x + D;
            const double pp = (A12 * x + B6) * x + C2;
            step = p * (double)rcp_approx_f32((float)pp);
            x -= step;
        }
        if (fabs(step) <= 1.0e-12 * (fabs(x) + 1.0)) return clampd(x, lo, hi);
    }
    return quartic_min64(A, B, C, D, lo, hi, paper_mode);
}

// ---------------------------------------------------------------------------
// Packed pair variant: the two columns of a vector in one float2, on the
// paired FP32 instructions (FADD2 / FMUL2 / FFMA2: two lanes per issue, the
// same rounding per lane as the scalar operations).  The common cases run
// packed: both lanes quadratic (A = 0), or both lanes on the Cardano branch
// with the discriminant's sign certified.  Any other combination (trig or
// uncertain branch, mixed A = 0 / A > 0, non-finite intermediate) is solved
// lane by lane by quartic_min32, so each lane gets the branch Algorithm 1
// gives it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.0f, -1.0f)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

// Newton step of newton_polish32 on both lanes.
__device__ __forceinline__ float2 newton_polish32x2(float2 A, float2 B, float2 C, float2 D, float2 x)
{
    const float2 A4 = mul2(splat2(4.0f), A), B3 = mul2(splat2(3.0f), B), C2 = add2(C, C);
    const float2 fp = fma2(fma2(fma2(A4, x, B3), x, C2), x, D);
    const float2 fpp = fma2(fma2(mul2(splat2(12.0f), A), x, mul2(splat2(6.0f), B)), x, C2);
    const float2 r = make_float2(rcp_fast(fpp.x), rcp_fast(fpp.y)); // used only where fpp > 0
    const float2 dx = mul2(fp, r);
    const float2 xn = sub2(x, dx);
    const float2 lim = mul2(splat2(0.0625f), add2(abs2(x), splat2(1.0f)));
    return make_float2((fpp.x > 0.0f && fabsf(dx.x) <= lim.x) ? xn.x : x.x,
                       (fpp.y > 0.0f && fabsf(dx.y) <= lim.y) ? xn.y : x.y);
}

// Lane by lane (out of line: the rare path stays out of the element loop).
static __device__ __noinline__ float2 quartic_min32_lanes(float2 A, float2 B, float2 C, float2 D, float2 lo,
                                                          float2 hi, int paper_mode, unsigned *esc)
{
    unsigned e = *esc;
    const float2 x = make_float2(quartic_min32(A.x, B.x, C.x, D.x, lo.x, hi.x, paper_mode, e),
                                 quartic_min32(A.y, B.y, C.y, D.y, lo.y, hi.y, paper_mode, e));
    *esc = e;
    return x;
}

__device__ __forceinline__ float2 quartic_min32x2(float2 A, float2 B, float2 C, float2 D, float2 lo, float2 hi,
                                                  int paper_mode, unsigned &esc)
{
#ifndef ADMM_COMPENSATED_POLISH
    if (A.x > 0.0f && A.y > 0.0f) {
        const float2 inv = make_float2(rcp_fast(A.x), rcp_fast(A.y));
        const float2 b = mul2(mul2(splat2(0.75f), B), inv);
        const float2 c = mul2(mul2(splat2(0.5f), C), inv);
        const float2 d = mul2(mul2(splat2(0.25f), D), inv);
        const float2 b3 = mul2(b, splat2(1.0f / 3.0f));
        const float2 b3s = mul2(b3, b3), b3c = mul2(b3s, b3);
        const float2 Q = fma2(c, splat2(1.0f / 3.0f), neg2(b3s));
        const float2 hc = mul2(splat2(0.5f), c);
        const float2 bhc = mul2(b3, hc);
        const float2 R = sub2(sub2(bhc, b3c), mul2(splat2(0.5f), d));
        const float2 Qs = mul2(Q, Q);
        const float2 Q3 = mul2(Qs, Q), R2 = mul2(R, R);
        const float2 Dl = add2(Q3, R2);
        // the forward error bound of quartic_min32, on both lanes
        const float2 mQ = fma2(abs2(c), splat2(1.0f / 3.0f), b3s);
        const float2 mR = fma2(splat2(0.5f), abs2(d), add2(abs2(bhc), abs2(b3c)));
        const float2 bound = mul2(splat2(7.68e-6f), fma2(Qs, mQ, mul2(abs2(R), mR)));
        if (Dl.x > bound.x && Dl.y > bound.y) { // Cardano on both lanes
            // here Delta > bound >= 0, so sqrt(Delta) > 0, |R +- sqrt(Delta)| > 0 and S != 0: the
            // zero guards of sqrt_fast, cbrt_fast and the T reciprocal are not needed (an S that
            // underflows gives a non-finite x and the lane-by-lane path below)
            const float2 sq = mul2(Dl, make_float2(rsqrtf(Dl.x), rsqrtf(Dl.y)));
            const float2 v = add2(R, make_float2(R.x >= 0.0f ? sq.x : -sq.x, R.y >= 0.0f ? sq.y : -sq.y));
            const float2 S = make_float2(copysignf(exp2f(__log2f(fabsf(v.x)) * (1.0f / 3.0f)), v.x),
                                         copysignf(exp2f(__log2f(fabsf(v.y)) * (1.0f / 3.0f)), v.y));
            const float2 rS = make_float2(rcp_fast(S.x), rcp_fast(S.y));
            const float2 T = mul2(neg2(Q), rS);
            const float2 x = newton_polish32x2(A, B, C, D, sub2(add2(S, T), b3));
            if (isfinite(x.x) && isfinite(x.y))
                return make_float2(clampf(x.x, lo.x, hi.x), clampf(x.y, lo.y, hi.y));
        }
    }
    if (A.x == 0.0f && A.y == 0.0f) { // quadratic on both lanes
        const float2 C2 = add2(C, C);
        const float2 x = mul2(neg2(D), make_float2(rcp_fast(C2.x), rcp_fast(C2.y)));
        return make_float2(clampf(x.x, lo.x, hi.x), clampf(x.y, lo.y, hi.y));
    }
#endif
    return quartic_min32_lanes(A, B, C, D, lo, hi, paper_mode, &esc);
}

} // namespace admm_impl

// Quartic minimiser in FP64: Algorithm 1 (Sec. III-B) and the projection of
// step (a) of the ADMM iteration (App. A).
//
// minimise A x^4 + B x^3 + C x^2 + D x over [lo, hi], A >= 0 (A = 0 needs C > 0).
// The extrema solve the monic cubic x^3 + b x^2 + c x + d with
// b = 3B/4A, c = C/2A, d = D/4A, classified by Q = c/3 - b^2/9,
// R = bc/6 - b^3/27 - d/2, Delta = Q^3 + R^2:
//   Delta > 0   one real root, Cardano: S + T - b/3 (stable pair: S from
//               R + sgn(R) sqrt(Delta), T = -Q/S, equal to the printed S, T);
//   Q = R = 0   triple root -b/3 (Vieta);
//   otherwise   three real roots 2 sqrt(-Q) cos((theta + 2 pi l)/3) - b/3 with
//               theta = acos(R / sqrt(-Q^3)).  For theta in [0, pi] the l = 1
//               root is the smallest and the l = 0 root the largest, so no
//               sort is needed; one sincos of theta/3 gives both, since
//               cos(t + 2pi/3) = -cos(t)/2 - (sqrt(3)/2) sin(t).
// The middle root is a maximiser.  The minimiser is the root with the lower
// value of F(x) = x^4/4 + (b/3) x^3 + (c/2) x^2 + d x (delta-f of Algorithm 1;
// F is the quartic divided by 4A).  Exact mode clamps both candidate roots
// to [lo, hi] before comparing (the constrained minimiser is always one of
// the two clamped roots); paper mode clamps the winner (Pi(argmin)).
// A tie keeps the smaller root, as Algorithm 1's else branch does.
//
// FP64 arithmetic is the scarce resource on this GPU (1/64 of the FP32 rate),
// so the two divisions and the cube root of the Cardano branch use FP32
// seeds from the special-function unit followed by FP64 Newton steps
// instead of the library routines: about a third of the FP64 instructions
// of the element update.  Each result is within a few ulp of the correctly
// rounded one.
#pragma once
#include "common.cuh"

namespace admm_impl {

__device__ __forceinline__ float rcp_approx_f32(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// 1/a: FP32 seed (relative error below 2^-22), then two Newton steps
// r <- r + r (1 - a r), each squaring the relative error.  Operands outside
// the FP32 normal range take the FP64 division.
__device__ __forceinline__ double rcp64(double a)
{
    const double aa = fabs(a);
    if (!(aa > 1e-30 && aa < 1e30)) return 1.0 / a;
    double r = (double)rcp_approx_f32((float)a);
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}

// S = cbrt(v) and 1/S for v != 0.  Seed w ~ |v|^(-1/3) from the FP32
// log2/exp2 units (relative error below 2e-5 over the accepted range), then
// two Newton steps on f(w) = w^-3 - |v|, w <- w (4 - |v| w^3) / 3; with
// w = w*(1 + e) the new error is about -2 e^2.  Operands outside the FP32
// normal range take the library cube root.
__device__ __forceinline__ void cbrt_rcbrt64(double v, double &S, double &invS)
{
    const double av = fabs(v);
    if (!(av > 1e-30 && av < 1e30)) {
        S = cbrt(v);
        invS = 1.0 / S;
        return;
    }
    float l, wf;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"((float)av));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(wf) : "f"(l * (-1.0f / 3.0f)));
    double w = (double)wf;
    w = w * fma(-av, w * w * w, 4.0) * (1.0 / 3.0);
    w = w * fma(-av, w * w * w, 4.0) * (1.0 / 3.0);
    S = copysign(av * w * w, v);
    invS = copysign(w, v);
}

__device__ __forceinline__ double delta_f64(double u, double v, double b, double c, double d)
{
    double u2 = u * u, v2 = v * v;
    return 0.25 * (u2 * u2 - v2 * v2) + (b * (1.0 / 3.0)) * (u2 * u - v2 * v) + (0.5 * c) * (u2 - v2) + d * (u - v);
}

// Returns the minimiser; *branch (if non-null) gets 0 Cardano, 1 triple,
// 2 trig, 3 quadratic.
__device__ __forceinline__ double quartic_min64(double A, double B, double C, double D, double lo,
                                                double hi, int paper_mode)
{
    if (A == 0.0)
        return clampd(-D * rcp64(2.0 * C), lo, hi);
    double inv = rcp64(A);
    double b = 0.75 * B * inv, c = 0.5 * C * inv, d = 0.25 * D * inv;
    double b3 = b * (1.0 / 3.0);
    double Q = c * (1.0 / 3.0) - b3 * b3;
    double R = b3 * (0.5 * c) - b3 * b3 * b3 - 0.5 * d;
    double Q3 = Q * Q * Q;
    double Dl = Q3 + R * R;
    if (Dl > 0.0) {
        double sq = sqrt(Dl);
        double S, invS;
        cbrt_rcbrt64(R >= 0.0 ? R + sq : R - sq, S, invS);
        double T = -Q * invS;
        return clampd(S + T - b3, lo, hi);
    }
    if (Q == 0.0 && R == 0.0)
        return clampd(-b3, lo, hi);
    double arg = clampd(R * rsqrt(-Q3), -1.0, 1.0);
    double t = acos(arg) * (1.0 / 3.0);
    double st, ct;
    sincos(t, &st, &ct);
    double two_sq = 2.0 * sqrt(-Q);
    double x3 = two_sq * ct - b3;                                        // largest root
    double x1 = two_sq * (-0.5 * ct - 0.86602540378443864676 * st) - b3; // smallest root
    if (paper_mode) {
        double xs = delta_f64(x1, x3, b, c, d) > 0.0 ? x3 : x1;
        return clampd(xs, lo, hi);
    }
    double u = clampd(x1, lo, hi), v = clampd(x3, lo, hi);
    return delta_f64(u, v, b, c, d) > 0.0 ? v : u;
}

} // namespace admm_impl

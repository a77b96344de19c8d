// Mixed-precision element work shared by the single-instance and batched
// solve kernels: step (a) of App. A for all sources of a few consecutive
// columns in FP32 (Algorithm 1 through quartic32.cuh), steps (e) and (f) on
// the float-float column state, and the float-float accumulation of the
// capacity sums over k.
#pragma once
#include "common.cuh"
#include "internal.h"
#include "quartic32.cuh"

namespace admm_impl {

// ---------------------------------------------------------------------------
// Mixed phase 1: a float4 quad of columns (j, k0..k0+3), FP32 element work.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg((const float4 *)p); }
__device__ __forceinline__ float4 ld4(const float *p) { return *(const float4 *)p; }
__device__ __forceinline__ float f4(const float4 &v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w)); }

// g = b2 x^2 + b1 x as an unevaluated sum hi + lo (error-free products and sum).
__device__ __forceinline__ void g_ff(float b2, float b1, float x, float &hi, float &lo)
{
    const float x2 = x * x;
    const float ex2 = __fmaf_rn(x, x, -x2);
    const float p = __fmul_rn(b2, x2);
    const float ep = __fmaf_rn(b2, x2, -p) + b2 * ex2;
    const float r = __fmul_rn(b1, x);
    const float er = __fmaf_rn(b1, x, -r);
    const float s = __fadd_rn(p, r);
    const float bb = __fsub_rn(s, p);
    const float es = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(r, bb));
    hi = s;
    lo = es + ep + er;
}

// (hi, lo) += (a, a_lo) in float-float.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float a, float a_lo)
{
    const float s = __fadd_rn(hi, a);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
    hi = s;
    lo = lo + (e + a_lo);
}

// Float-float arithmetic for the column state s, mu (steps (e), (f)).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_norm(float hi, float lo)
{
    const float s = __fadd_rn(hi, lo);
    return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const FF t = ff_two_sum(a.hi, b.hi);
    return ff_norm(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF ff_addf(FF a, float b)
{
    const FF t = ff_two_sum(a.hi, b);
    return ff_norm(t.hi, __fadd_rn(t.lo, a.lo));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// VW consecutive columns per thread (VW = 2 or 4), loaded as one vector.
template <int VW> __device__ __forceinline__ void ldv(const float *p, float *v, bool ro)
{
    if constexpr (VW == 4) {
        const float4 t = ro ? __ldg((const float4 *)p) : *(const float4 *)p;
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const float2 t = ro ? __ldg((const float2 *)p) : *(const float2 *)p;
        v[0] = t.x; v[1] = t.y;
    }
}
template <int VW> __device__ __forceinline__ void stv(float *p, const float *v)
{
    if constexpr (VW == 4) *(float4 *)p = make_float4(v[0], v[1], v[2], v[3]);
    else *(float2 *)p = make_float2(v[0], v[1]);
}

// Storage of one instance for the mixed element update (FP32 arrays with
// row stride ld; s, mu float-float as hi and lo arrays).
struct ElemF32 {
    const float *f2, *f1, *g2, *g1, *g0, *lo, *hi, *y;
    float *x, *s, *mu, *s_lo, *mu_lo;
    int n, m, q, ld, sweep, xmin_mode;
};

// L2 prefetch of everything vec32 reads for the columns (j, k0..): issued
// one vector ahead, so the loads of the next vector hit L2 instead of
// waiting on HBM.  Prefetches are hints and touch only rows the update reads.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <int M>
__device__ __forceinline__ void prefetch_vec32(const ElemF32 &a, int j, int k0, bool cold)
{
    const size_t col = (size_t)j * a.ld + k0;
    prefetch_l2(a.y + col);
    prefetch_l2(a.s + col);
    prefetch_l2(a.mu + col);
    prefetch_l2(a.s_lo + col);
    prefetch_l2(a.mu_lo + col);
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < a.m) {
            const size_t e = ((size_t)i * a.q + j) * a.ld + k0;
            prefetch_l2(a.x + e);
            prefetch_l2(a.f2 + e);
            prefetch_l2(a.f1 + e);
            prefetch_l2(a.g2 + e);
            prefetch_l2(a.g1 + e);
            if (cold) prefetch_l2(a.g0 + e);
            prefetch_l2(a.lo + (size_t)i * a.ld + k0);
            prefetch_l2(a.hi + (size_t)i * a.ld + k0);
        }
}

// Step (a) for all sources of VW columns (j, k0..k0+VW-1), then (e), (f).
// uoff[pr] = zeta + lambda of pair pr in FP32; x1 and nu are the FP64 pair
// scalars (read at k = 0 only).  rec (if k0 == 0) receives x at k = 0.
template <int M, int VW, bool C64>
__device__ __forceinline__ void vec32(const ElemF32 &a, const float *uoff, const double *x1s, const double *nus,
                                      int j, int k0, bool check, bool cold, float mu_div, float rho1, float rho3,
                                      float rho4, float iq, float *ghi, float *glo, float *dmx, float *dmn,
                                      float &cm_r, float &cm_s, unsigned &esc, double *rec)
{
    const int m = a.m, q = a.q, ld = a.ld, n = a.n;
    const float *__restrict__ F2 = a.f2;
    const float *__restrict__ F1 = a.f1;
    const float *__restrict__ G2 = a.g2;
    const float *__restrict__ G1 = a.g1;
    const float *__restrict__ G0 = a.g0;
    const float *__restrict__ LO = a.lo;
    const float *__restrict__ HI = a.hi;
    const float *__restrict__ Y = a.y;
    float *X = a.x, *Sv = a.s, *MU = a.mu;
    float *SL = a.s_lo, *ML = a.mu_lo;

    const size_t col = (size_t)j * ld + k0;
    float yv[VW], st[VW], mu[VW], stl[VW], mul[VW];
    ldv<VW>(Y + col, yv, true);
    ldv<VW>(Sv + col, st, false);
    ldv<VW>(MU + col, mu, false);
    ldv<VW>(SL + col, stl, false);
    ldv<VW>(ML + col, mul, false);
    if (mu_div != 1.0f) {
#pragma unroll
        for (int c = 0; c < VW; ++c) {
            mu[c] = mu[c] / mu_div;
            mul[c] = mul[c] / mu_div;
        }
    }
    float xt[M][VW], xs[M][VW];
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            ldv<VW>(X + ((size_t)i * q + j) * ld + k0, xt[i], false);
#pragma unroll
            for (int c = 0; c < VW; ++c) xs[i][c] = xt[i][c];
        }
    bool valid[VW];
#pragma unroll
    for (int c = 0; c < VW; ++c) valid[c] = k0 + c < n;
    const bool jac = a.sweep == ADMM_JACOBI;
    // sum of x over the sources: Gauss-Seidel keeps it current as the sweep
    // replaces x_i, Jacobi keeps the previous iterate's
    float xsum[VW];
#pragma unroll
    for (int c = 0; c < VW; ++c) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < m) t += xt[i][c];
        xsum[c] = t;
    }

#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (i < m) {
            const size_t e = ((size_t)i * q + j) * ld + k0;
            float A2[VW], A1[VW], B2[VW], B1[VW], L4[VW], H4[VW], Z4[VW];
            ldv<VW>(F2 + e, A2, true);
            ldv<VW>(F1 + e, A1, true);
            ldv<VW>(G2 + e, B2, true);
            ldv<VW>(G1 + e, B1, true);
            ldv<VW>(LO + (size_t)i * ld + k0, L4, true);
            ldv<VW>(HI + (size_t)i * ld + k0, H4, true);
            if (cold) ldv<VW>(G0 + e, Z4, true);
            else {
#pragma unroll
                for (int c = 0; c < VW; ++c) Z4[c] = 0.0f;
            }
            const int pr = i * q + j;
            const float uo = uoff[pr];
#pragma unroll
            for (int c = 0; c < VW; ++c) {
                const float a2 = A2[c], a1 = A1[c], b2 = B2[c], b1 = B1[c], g0 = Z4[c];
                const float x0 = xt[i][c];
                const float gq_old = (b2 * x0 + b1) * x0;
                const float u = cold ? -g0 : gq_old + uo;
                const float others = xsum[c] - x0; // sum over l != i (x_i is still x0 here)
                const float phi = ((st[c] - others) + yv[c]) + mu[c];
                const float A = 0.5f * rho1 * b2 * b2;
                const float B = rho1 * b2 * b1;
                float C = a2 * iq + 0.5f * rho1 * (b1 * b1 - 2.0f * b2 * u) + 0.5f * rho3;
                float D = a1 * iq - rho1 * b1 * u - rho3 * phi;
                if (k0 + c == 0) {
                    C += 0.5f * rho4;
                    D -= rho4 * (float)(x1s[i] + nus[pr]);
                }
                const float xn = C64 ? quartic_min_fp64cubic(A, B, C, D, L4[c], H4[c], a.xmin_mode)
                                     : quartic_min32(A, B, C, D, L4[c], H4[c], a.xmin_mode, esc);
                if (!jac) xsum[c] += xn - x0;
                xs[i][c] = xn;
                if (valid[c]) {
                    float ghh, gll;
                    g_ff(b2, b1, xn, ghh, gll);
                    ff_add(ghi[i], glo[i], ghh, gll);
                    if (check) {
                        const float dk = cold ? ghh + g0 : ghh - gq_old;
                        dmx[i] = fmaxf(dmx[i], dk);
                        dmn[i] = fminf(dmn[i], dk);
                    }
                }
            }
        }
    }
    // (e), (f) in float-float: the column state carries about 48 bits, so
    // mu's accumulation of ever smaller primal residuals is not lost to FP32
    // rounding and the dual residual term of s settles below 1e-6.
    float sn[VW], snl[VW], mn[VW], mnl[VW];
#pragma unroll
    for (int c = 0; c < VW; ++c) {
        FF sx = {0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < m) sx = ff_addf(sx, xs[i][c]);
        const FF muf = {mu[c], mul[c]}, stf = {st[c], stl[c]};
        const FF v = ff_add(ff_addf(sx, -yv[c]), ff_neg(muf));       // sum_i x - y - mu
        const FF sv = v.hi > 0.0f ? v : FF{0.0f, 0.0f};               // (e)
        const FF t = ff_addf(ff_add(sv, ff_neg(sx)), yv[c]);          // s - sum_i x + y
        const FF mnew = ff_add(muf, t);                                // (f)
        sn[c] = sv.hi;
        snl[c] = sv.lo;
        mn[c] = mnew.hi;
        mnl[c] = mnew.lo;
        if (check && valid[c]) {
            cm_r = fmaxf(cm_r, fabsf(t.hi + t.lo));
            FF dx = {0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (i < m) dx = ff_add(dx, ff_two_sum(xs[i][c], -xt[i][c]));
            const FF d = ff_add(ff_add(sv, ff_neg(stf)), ff_neg(dx));  // s - s~ - sum_i (x - x~)
            cm_s = fmaxf(cm_s, fabsf(d.hi + d.lo));
        }
    }
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) stv<VW>(X + ((size_t)i * q + j) * ld + k0, xs[i]);
    stv<VW>(Sv + col, sn);
    stv<VW>(MU + col, mn);
    stv<VW>(SL + col, snl);
    stv<VW>(ML + col, mnl);
    if (k0 == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < m) rec[i * 4 + 3] = (double)xs[i][0];
    }
}


} // namespace admm_impl

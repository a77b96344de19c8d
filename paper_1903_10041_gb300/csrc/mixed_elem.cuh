// Mixed-precision element work shared by the single-instance and batched
// solve kernels: step (a) of App. A for all sources of a pair of consecutive
// columns in FP32 (Algorithm 1 through quartic32.cuh), steps (e) and (f) on
// the float-float column state, and the float-float accumulation of the
// capacity sums over k.  The two columns travel as one float2 through the
// paired FP32 instructions.
#pragma once
#include "common.cuh"
#include "internal.h"
#include "quartic32.cuh"

namespace admm_impl {

// Float-float arithmetic (segment reductions of the capacity sums).
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

// Storage of one instance for the mixed element update (FP32 arrays with
// row stride ld; s, mu float-float as hi and lo arrays).  The instance's
// ranges start at element oe (x and coefficients), ob (bounds) and oc
// (columns) of the arrays.  IX is the index type: size_t for a single
// instance of any size; unsigned for the batched kernel, whose arrays hold
// at most 2^32 - 1 elements, so that an address is the array's base (a
// kernel parameter) plus one 32-bit index and no per-instance 64-bit
// pointers stay live in registers.
template <class IX> struct ElemF32T {
    const float *f2, *f1, *g2, *g1, *g0, *lo, *hi, *y;
    float *x, *s, *mu, *s_lo, *mu_lo;
    int n, m, q, ld, sweep, xmin_mode;
    int cq, cj; // coefficient row of pair (i, j): i * cq + j * cj
    unsigned long long *dbg = nullptr; // bounds record (checked builds)
    IX oe = 0, ob = 0, oc = 0;
    // lengths of the instance's ranges: columns [q][ld], x [m][q][ld],
    // coefficients [m][ld] when shared else [m][q][ld], bounds [m][ld]
    __device__ __forceinline__ size_t len_col() const { return (size_t)q * ld; }
    __device__ __forceinline__ size_t len_x() const { return (size_t)m * q * ld; }
    __device__ __forceinline__ size_t len_coef() const { return (size_t)m * (cj ? q : 1) * ld; }
    __device__ __forceinline__ size_t len_bound() const { return (size_t)m * ld; }
    // array indices of the column pair (j, k0): column arrays, x of source i,
    // coefficients of source i, bounds of source i (checked in the instance's range)
    __device__ __forceinline__ IX col(int j, int k0) const
    {
        return oc + (IX)ADMM_IDX((IX)j * ld + k0, 2, len_col(), dbg, DBG_COL);
    }
    __device__ __forceinline__ IX xe(int i, int j, int k0) const
    {
        return oe + (IX)ADMM_IDX(((IX)i * q + j) * ld + k0, 2, len_x(), dbg, DBG_X);
    }
    __device__ __forceinline__ IX ce(int i, int j, int k0) const
    {
        return oe + (IX)ADMM_IDX(((IX)i * cq + (IX)j * cj) * ld + k0, 2, len_coef(), dbg, DBG_COEF);
    }
    __device__ __forceinline__ IX be(int i, int k0) const
    {
        return ob + (IX)ADMM_IDX((IX)i * ld + k0, 2, len_bound(), dbg, DBG_BOUND);
    }
};
using ElemF32 = ElemF32T<size_t>;

// L2 prefetch of everything vec32 reads for the columns (j, k0..): issued
// one vector ahead, so the loads of the next vector hit L2 instead of
// waiting on HBM.  Prefetches are hints and touch only rows the update reads.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <int M, class EA> __device__ __forceinline__ void prefetch_vec32(const EA &a, int j, int k0, bool cold)
{
    const auto col = a.col(j, k0);
    prefetch_l2(a.y + col);
    prefetch_l2(a.s + col);
    prefetch_l2(a.mu + col);
    prefetch_l2(a.s_lo + col);
    prefetch_l2(a.mu_lo + col);
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < a.m) {
            const auto e = a.xe(i, j, k0);
            const auto ec = a.ce(i, j, k0);
            const auto eb = a.be(i, k0);
            prefetch_l2(a.x + e);
            prefetch_l2(a.f2 + ec);
            prefetch_l2(a.f1 + ec);
            prefetch_l2(a.g2 + ec);
            prefetch_l2(a.g1 + ec);
            if (cold) prefetch_l2(a.g0 + ec);
            prefetch_l2(a.lo + eb);
            prefetch_l2(a.hi + eb);
        }
}

// Shared-memory staging of the read-only coefficients (batched kernel):
// each lane copies the f2, f1, g2, g1 of every source and y of its next
// column pair into its own slots of a per-warp stage with 8-byte cp.async
// copies, one pair ahead, and reads the current pair from the other stage.
// A lane reads only the slots it filled, so cp.async.wait_group orders it;
// no other synchronisation is needed.  Slot s of a stage holds 32 float2
// (one per lane): slot 0 y, slots 1 + 4 i + {0, 1, 2, 3} f2, f1, g2, g1 of
// source i.
template <int M> __host__ __device__ constexpr int stage_slots() { return 4 * M + 1; }
__device__ __forceinline__ void cp_async8(float2 *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies the staged arrays of the column pair (j, k0) into the lane's slots
// (dst = stage base + lane).
template <int M, class EA> __device__ __forceinline__ void stage_vec32(const EA &a, int j, int k0, float2 *dst)
{
    cp_async8(dst, a.y + a.col(j, k0));
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < a.m) {
            const auto d = a.ce(i, j, k0);
            cp_async8(dst + (1 + 4 * i) * 32, a.f2 + d);
            cp_async8(dst + (2 + 4 * i) * 32, a.f1 + d);
            cp_async8(dst + (3 + 4 * i) * 32, a.g2 + d);
            cp_async8(dst + (4 + 4 * i) * 32, a.g1 + d);
        }
}

// Rolling staging (batched kernel, launches whose instances stay on one team):
// every array the element update reads comes through the lane's own slots of
// one per-warp stage, each slot group refilled for the next column pair right
// after it is read.  Slots: 0 y, 1 s, 2 mu, 3 s_lo, 4 mu_lo, 5 + i x of source
// i (the column group), then 5 + M + 6 i + {0..5} f2, f1, g2, g1, lo, hi of
// source i.  A pair's copies are committed as 1 + M groups (column, then one
// per source slot, empty past m), so the group a step needs is always the
// oldest but M: every wait is cp.async.wait_group M.  The copies cache in L1
// (8-byte cp.async has no L2-only form), so the mode is for launches where no
// instance moves to another SM: its own L1 never holds lines another SM wrote.
template <int M> __host__ __device__ constexpr int roll_slots() { return 5 + 7 * M; }
// Slots per warp of the batched kernel's stage region (either staging mode).
template <int M> __host__ __device__ constexpr int stage_region_slots()
{
    return 2 * stage_slots<M>() > roll_slots<M>() ? 2 * stage_slots<M>() : roll_slots<M>();
}
template <int M> __device__ __forceinline__ void cp_async_wait_m()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(M) : "memory");
}
template <int M, class EA> __device__ __forceinline__ void roll_issue_col(const EA &a, int j, int k0, float2 *dst)
{
    const auto col = a.col(j, k0);
    cp_async8(dst + 0 * 32, a.y + col);
    cp_async8(dst + 1 * 32, a.s + col);
    cp_async8(dst + 2 * 32, a.mu + col);
    cp_async8(dst + 3 * 32, a.s_lo + col);
    cp_async8(dst + 4 * 32, a.mu_lo + col);
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < a.m) cp_async8(dst + (5 + i) * 32, a.x + a.xe(i, j, k0));
}
template <int M, class EA>
__device__ __forceinline__ void roll_issue_src(const EA &a, int i, int j, int k0, float2 *dst)
{
    const auto d = a.ce(i, j, k0);
    const auto eb = a.be(i, k0);
    float2 *p = dst + (5 + M + 6 * i) * 32;
    cp_async8(p + 0 * 32, a.f2 + d);
    cp_async8(p + 1 * 32, a.f1 + d);
    cp_async8(p + 2 * 32, a.g2 + d);
    cp_async8(p + 3 * 32, a.g1 + d);
    cp_async8(p + 4 * 32, a.lo + eb);
    cp_async8(p + 5 * 32, a.hi + eb);
}
// The copies of a piece's first column pair (any: the lane has one).
template <int M, class EA>
__device__ __forceinline__ void roll_prologue(const EA &a, int j, int k0, bool any, float2 *stg)
{
    if (any) roll_issue_col<M>(a, j, k0, stg);
    cp_async_commit();
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (any && i < a.m) roll_issue_src<M>(a, i, j, k0, stg);
        cp_async_commit();
    }
}

// L2 prefetch of what the staged element update still reads from global
// memory: x, the bounds and the column state s, mu.
template <int M, class EA> __device__ __forceinline__ void prefetch_mutable(const EA &a, int j, int k0)
{
    const auto col = a.col(j, k0);
    prefetch_l2(a.s + col);
    prefetch_l2(a.mu + col);
    prefetch_l2(a.s_lo + col);
    prefetch_l2(a.mu_lo + col);
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < a.m) {
            prefetch_l2(a.x + a.xe(i, j, k0));
            const auto eb = a.be(i, k0);
            prefetch_l2(a.lo + eb);
            prefetch_l2(a.hi + eb);
        }
}

// Float-float on packed pairs (the two columns of a vector).
struct FF2 {
    float2 hi, lo;
};
__device__ __forceinline__ FF2 ff2_two_sum(float2 a, float2 b)
{
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ FF2 ff2_norm(float2 hi, float2 lo)
{
    const float2 s = add2(hi, lo);
    return {s, sub2(lo, sub2(s, hi))};
}
__device__ __forceinline__ FF2 ff2_add(FF2 a, FF2 b)
{
    const FF2 t = ff2_two_sum(a.hi, b.hi);
    return ff2_norm(t.hi, add2(t.lo, add2(a.lo, b.lo)));
}
__device__ __forceinline__ FF2 ff2_addf(FF2 a, float2 b)
{
    const FF2 t = ff2_two_sum(a.hi, b);
    return ff2_norm(t.hi, add2(t.lo, a.lo));
}
__device__ __forceinline__ FF2 ff2_neg(FF2 a) { return {neg2(a.hi), neg2(a.lo)}; }

// g = b2 x^2 + b1 x as hi + lo on both lanes (error-free products and sum).
__device__ __forceinline__ void g_ff2(float2 b2, float2 b1, float2 x, float2 &hi, float2 &lo)
{
    const float2 x2 = mul2(x, x);
    const float2 ex2 = fma2(x, x, neg2(x2));
    const float2 p = mul2(b2, x2);
    const float2 ep = fma2(b2, ex2, fma2(b2, x2, neg2(p)));
    const float2 r = mul2(b1, x);
    const float2 er = fma2(b1, x, neg2(r));
    const float2 s = add2(p, r);
    const float2 bb = sub2(s, p);
    const float2 es = add2(sub2(p, sub2(s, bb)), sub2(r, bb));
    hi = s;
    lo = add2(add2(es, ep), er);
}

// (hi, lo) += (a, a_lo) lane by lane in float-float.
__device__ __forceinline__ void ff2_acc(float2 &hi, float2 &lo, float2 a, float2 a_lo)
{
    const float2 s = add2(hi, a);
    const float2 bb = sub2(s, hi);
    const float2 e = add2(sub2(hi, sub2(s, bb)), sub2(a, bb));
    hi = s;
    lo = add2(lo, add2(e, a_lo));
}

// Mutable state (x, s, mu) bypasses L1: in round-robin launches an instance
// can move to another SM, whose L1 may hold lines of an earlier pass.
__device__ __forceinline__ float2 ld2(const float *p) { return __ldcg((const float2 *)p); }
__device__ __forceinline__ float2 ldg2(const float *p) { return __ldg((const float2 *)p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *(float2 *)p = v; }

// Step (a) for all sources of the column pair (j, k0), (j, k0 + 1), then
// (e), (f), on packed pairs.  uoff[pr] = zeta + lambda and x1nu[pr] =
// x1 + nu (read at k = 0 only) of pair pr, rounded to FP32 once per
// iteration by the caller, so no FP64 operation runs per element.  The capacity
// sums accumulate per lane in ghi/glo (the caller combines the lanes), the
// D_k extrema in dmx/dmn.  rec (if k0 == 0) receives x at k = 0 as an FP32
// value in the first four bytes of its slot (the scalar phase widens it).
// STAGE_ROLL: the inputs come from the lane's rolling stage stg, and each slot
// group is refilled with the pair k0n (if >= 0) as soon as it is read.  The
// first column is always < n; the second may be padding (k0 + 1 = n), and
// then takes no part in the sums and residuals.
// Where vec32 reads its inputs: global memory, the double stage of
// stage_vec32 (coefficients and y), or the rolling stage (everything).
enum { STAGE_NONE = 0, STAGE_DOUBLE = 1, STAGE_ROLL = 2 };

template <int M, int VW, bool C64, int STAGE = STAGE_NONE, class EA>
__device__ __forceinline__ void vec32(const EA &a, const float *uoff, const float *x1nu,
                                      int j, int k0, bool check, bool cold, float mu_div, float rho1, float rho3,
                                      float rho4, float iq, float2 *ghi, float2 *glo, float *dmx, float *dmn,
                                      float &cm_r, float &cm_s, unsigned &esc, double *rec,
                                      float2 *stg = nullptr, int k0n = -1)
{
    static_assert(VW == 2, "the element update works on column pairs");
    constexpr bool ROLL = STAGE == STAGE_ROLL;
    const int m = a.m, q = a.q, n = a.n;
    const auto col = a.col(j, k0);
    if constexpr (ROLL) cp_async_wait_m<M>(); // the column group of this pair
    const float2 yv = STAGE != STAGE_NONE ? stg[0] : ldg2(a.y + col);
    const float2 st = ROLL ? stg[1 * 32] : ld2(a.s + col), stl = ROLL ? stg[3 * 32] : ld2(a.s_lo + col);
    float2 mu = ROLL ? stg[2 * 32] : ld2(a.mu + col), mul = ROLL ? stg[4 * 32] : ld2(a.mu_lo + col);
    if (mu_div != 1.0f) {
        mu = make_float2(mu.x / mu_div, mu.y / mu_div);
        mul = make_float2(mul.x / mu_div, mul.y / mu_div);
    }
    float2 xt[M];
    float2 xsum = splat2(0.0f); // sum of x over the sources, kept current by Gauss-Seidel
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            xt[i] = ROLL ? stg[(5 + i) * 32] : ld2(a.x + a.xe(i, j, k0));
            xsum = add2(xsum, xt[i]);
        }
    if constexpr (ROLL) { // the column group has been read: refill it for the next pair
        if (k0n >= 0) roll_issue_col<M>(a, j, k0n, stg);
        cp_async_commit();
    }
    const bool v1 = k0 + 1 < n;
    const bool jac = a.sweep == ADMM_JACOBI;
    const float2 h1 = splat2(0.5f * rho1), h3 = splat2(0.5f * rho3), iq2 = splat2(iq);
    const float2 nr1 = splat2(-rho1), nr3 = splat2(-rho3);
    FF2 sx = {splat2(0.0f), splat2(0.0f)}, dx = {splat2(0.0f), splat2(0.0f)};

#pragma unroll
    for (int i = 0; i < M; ++i) {
        if constexpr (ROLL) cp_async_wait_m<M>(); // source i's group of this pair
        if (i < m) {
            const auto e = a.ce(i, j, k0); // coefficient element
            const auto eb = a.be(i, k0);
            const float2 *sp = stg + (ROLL ? 5 + M + 6 * i : 1 + 4 * i) * 32;
            const float2 a2 = STAGE != STAGE_NONE ? sp[0] : ldg2(a.f2 + e);
            const float2 a1 = STAGE != STAGE_NONE ? sp[32] : ldg2(a.f1 + e);
            const float2 b2 = STAGE != STAGE_NONE ? sp[64] : ldg2(a.g2 + e);
            const float2 b1 = STAGE != STAGE_NONE ? sp[96] : ldg2(a.g1 + e);
            const float2 L = ROLL ? sp[128] : ldg2(a.lo + eb), H = ROLL ? sp[160] : ldg2(a.hi + eb);
            if constexpr (ROLL) {
                if (k0n >= 0) roll_issue_src<M>(a, i, j, k0n, stg);
                cp_async_commit();
            }
            const float2 g0 = cold ? ldg2(a.g0 + e) : splat2(0.0f);
            const int pr = i * q + j;
            const float2 x0 = xt[i];
            const float2 gq_old = mul2(fma2(b2, x0, b1), x0);
            const float2 u = cold ? neg2(g0) : add2(gq_old, splat2(uoff[pr]));
            const float2 others = sub2(xsum, x0); // sum over l != i (x_i is still x0 here)
            const float2 phi = add2(add2(sub2(st, others), yv), mu);
            const float2 hb2 = mul2(h1, b2); // (rho_1 / 2) b2; B = (rho_1 b2) b1 = hb2 (2 b1) exactly
            const float2 A = mul2(hb2, b2);
            const float2 B = mul2(hb2, add2(b1, b1));
            const float2 t = fma2(mul2(splat2(-2.0f), b2), u, mul2(b1, b1)); // b1^2 - 2 b2 u
            float2 C = fma2(a2, iq2, fma2(h1, t, h3));
            float2 D = fma2(a1, iq2, fma2(mul2(nr1, b1), u, mul2(nr3, phi)));
            if (k0 == 0) {
                C.x += 0.5f * rho4;
                D.x -= rho4 * x1nu[pr];
            }
            float2 xn;
            if constexpr (C64)
                xn = make_float2(quartic_min_fp64cubic(A.x, B.x, C.x, D.x, L.x, H.x, a.xmin_mode),
                                 quartic_min_fp64cubic(A.y, B.y, C.y, D.y, L.y, H.y, a.xmin_mode));
            else
                xn = quartic_min32x2(A, B, C, D, L, H, a.xmin_mode, esc);
            if (!jac) xsum = add2(xsum, sub2(xn, x0));
            sx = ff2_addf(sx, xn); // sum_i x of (e), (f) in source order
            if (check) dx = ff2_add(dx, ff2_two_sum(xn, neg2(x0)));
            st2(a.x + a.xe(i, j, k0), xn);
            if (k0 == 0) *(float *)(rec + i * 4 + 3) = xn.x; // FP32 in the slot; widened by the reader
            float2 ghh, gll;
            g_ff2(b2, b1, xn, ghh, gll);
            if (!v1) {
                ghh.y = 0.0f;
                gll.y = 0.0f;
            }
            ff2_acc(ghi[i], glo[i], ghh, gll);
            if (check) {
                const float2 dk = cold ? add2(ghh, g0) : sub2(ghh, gq_old);
                dmx[i] = fmaxf(dmx[i], v1 ? fmaxf(dk.x, dk.y) : dk.x);
                dmn[i] = fminf(dmn[i], v1 ? fminf(dk.x, dk.y) : dk.x);
            }
        } else if constexpr (ROLL) {
            cp_async_commit(); // the empty group of an unused source slot
        }
    }
    // (e), (f) in float-float: the column state carries about 48 bits, so
    // mu's accumulation of ever smaller primal residuals is not lost to FP32
    // rounding and the dual residual term of s settles below 1e-6.  With
    // d = sum_i x - y - mu, step (e) gives s = max(0, d) and step (f)
    // mu + s - sum_i x + y = s - d = max(0, -d): one float-float chain for d
    // gives both, and the residual mu_new - mu is formed on check iterations only.
    const FF2 muf = {mu, mul}, stf = {st, stl};
    const FF2 v = ff2_add(ff2_addf(sx, neg2(yv)), ff2_neg(muf));        // sum_i x - y - mu
    const FF2 sv = {make_float2(v.hi.x > 0.0f ? v.hi.x : 0.0f, v.hi.y > 0.0f ? v.hi.y : 0.0f),
                    make_float2(v.hi.x > 0.0f ? v.lo.x : 0.0f, v.hi.y > 0.0f ? v.lo.y : 0.0f)}; // (e)
    const FF2 nv = ff2_neg(v);
    const FF2 mnew = {make_float2(v.hi.x < 0.0f ? nv.hi.x : 0.0f, v.hi.y < 0.0f ? nv.hi.y : 0.0f),
                      make_float2(v.hi.x < 0.0f ? nv.lo.x : 0.0f, v.hi.y < 0.0f ? nv.lo.y : 0.0f)}; // (f)
    if (check) {
        const FF2 t = ff2_add(mnew, ff2_neg(muf)); // s - sum_i x + y
        const FF2 d = ff2_add(ff2_add(sv, ff2_neg(stf)), ff2_neg(dx)); // s - s~ - sum_i (x - x~)
        cm_r = fmaxf(cm_r, fabsf(t.hi.x + t.lo.x));
        cm_s = fmaxf(cm_s, fabsf(d.hi.x + d.lo.x));
        if (v1) {
            cm_r = fmaxf(cm_r, fabsf(t.hi.y + t.lo.y));
            cm_s = fmaxf(cm_s, fabsf(d.hi.y + d.lo.y));
        }
    }
    st2(a.s + col, sv.hi);
    st2(a.mu + col, mnew.hi);
    st2(a.s_lo + col, sv.lo);
    st2(a.mu_lo + col, mnew.lo);
}

// Lane sum of the per-thread capacity-sum accumulators of one source.
__device__ __forceinline__ FF lanes_sum(float2 hi, float2 lo) { return ff_add(ff_norm(hi.x, lo.x), ff_norm(hi.y, lo.y)); }

} // namespace admm_impl

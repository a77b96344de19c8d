// Persistent single-instance solve kernel: the whole ADMM loop of App. A on
// the device, one cooperative launch per solve.
//
// Work split.  The columns (j, k) are taken in j-major order and cut into
// one contiguous range per CTA of (nearly) equal length: either every row j
// cut into the same number of pieces (no CTA straddles two rows), or, for
// short rows, flat chunks of `chunk` columns, where the row segments of one
// CTA are worked on side by side by disjoint warps (or, when the segments are
// long, one after another by all warps).  The thread that owns a column
// updates all m sources of it in registers (step (a) sweeps the sources in
// order, so the Gauss-Seidel sums over l != i stay local), then steps (e)
// and (f) for that column.  The per-(i, j) sums over k that steps (b) and
// (d) and the residuals need are segmented reductions: each CTA reduces each
// row segment it owns (warp shuffles, then shared memory) into a partial
// record; after one grid barrier every CTA adds the records of each row in
// a fixed order and runs the per-(i, j) scalar steps (b), (c), (d), (g),
// (h), (i), the residuals and the stop test redundantly, so all CTAs hold
// identical scalars and take the same stop decision without a second
// barrier.  Partial records are double-buffered by iteration parity.
//
// Identities used (derived from steps (b) and (g)): after every iteration
// lambda^(i,j) is constant over k and z_k = g_k(x_k) + zeta with
// zeta = lambda_new - lambda_old, so theta_k = z_k + lambda =
// g_k(x~_k) + zeta + lambda needs no per-element z or lambda.  The zero start
// (z = 0, the paper's iteration from zeros) is flagged `cold`, where
// theta = 0 instead.
//
// Precision variants (template PREC):
//   ADMM_FP64             one column per thread, dense column space (rs = n);
//   ADMM_MIXED            FP32 storage and element work on column pairs
//                         (float2, paired FP32 instructions) over a padded
//                         column space (rs = ld); the
//                         capacity sums over k are accumulated per thread in
//                         float-float (about 48 bits) and reduced in FP64; the
//                         column state s, mu is stored and updated in
//                         float-float; the cubic's branch is decided as FP64
//                         would decide it;
//   ADMM_MIXED_FP64CUBIC  as ADMM_MIXED with the cubic step in FP64.
// The per-(i, j) scalar steps, residuals and stop test are FP64 in all three.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "mixed_elem.cuh"
#include "quartic64.cuh"

namespace admm_impl {

namespace {

struct Sm {
    double *lam, *zeta, *h, *p, *nu, *x1, *rho, *flags; // mirror of the scalar state
    double *x0;   // [mq]
    double *x1n;  // [kMaxM]
    double *red;  // [kSingleWarpsMax][kMaxM][3]
    double *mx;   // [kSingleWarpsMax][8]
    double *bc;   // [16] broadcast
    int *segof;   // [kSingleWarpsMax] segment (within the pass) of each warp
    float *uoff;  // [mq] zeta + lambda in FP32 (mixed variants)
    float *x1nu;  // [mq] x1 + nu in FP32 (mixed variants)
};

// Bytes of the shared state carve() lays out, rounded up to 16: the rolling
// stage of the mixed kernels (m <= 4) starts there.
__host__ __device__ inline size_t single_carve_bytes(int m, int q)
{
    const int mq = m * q;
    const size_t b = sizeof(double) * ((size_t)scal_size(m, q) + mq + kMaxM + kSingleWarpsMax * kMaxM * 3 +
                                       kSingleWarpsMax * 8 + 16 + kSingleWarpsMax) +
                     sizeof(float) * 2 * (size_t)mq;
    return (b + 15) / 16 * 16;
}

__device__ __forceinline__ Sm carve(double *base, int m, int q)
{
    const int mq = m * q;
    Sm s;
    s.lam = base;
    s.zeta = base + mq;
    s.h = base + 2 * mq;
    s.p = base + 3 * mq;
    s.nu = base + 4 * mq;
    s.x1 = base + 5 * mq;
    s.rho = s.x1 + m;
    s.flags = s.rho + 4;
    double *t = base + scal_size(m, q);
    s.x0 = t;
    t += mq;
    s.x1n = t;
    t += kMaxM;
    s.red = t;
    t += kSingleWarpsMax * kMaxM * 3;
    s.mx = t;
    t += kSingleWarpsMax * 8;
    s.bc = t;
    t += 16;
    s.segof = (int *)t;
    t += kSingleWarpsMax;
    s.uoff = (float *)t;
    s.x1nu = s.uoff + mq;
    return s;
}

// Block-wide max of up to 8 non-negative values; every thread gets the results in v[].
template <int NV, int NWP> __device__ __forceinline__ void block_max(double *v, const Sm &sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        double r = warp_max_nonneg(v[t]);
        if (lane == 0) sm.mx[w * 8 + t] = r;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double r = 0.0;
        for (int ww = 0; ww < NWP; ++ww) r = max_nonneg(r, sm.mx[ww * 8 + threadIdx.x]);
        sm.bc[threadIdx.x] = r;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = sm.bc[t];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// FP64 phase 1: step (a) for all sources of column (j, k), then (e), (f).
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void column64(const SingleArgs &a, const Sm &sm, int j, int k, bool check,
                                         bool cold, double mu_div, double *gs, double *dmx, double *dmn,
                                         double &cm_r, double &cm_s, double *rec)
{
    const int m = a.m, q = a.q, ld = a.ld;
    const double *F2 = (const double *)a.f2, *F1 = (const double *)a.f1;
    const double *G2 = (const double *)a.g2, *G1 = (const double *)a.g1, *G0 = (const double *)a.g0;
    const double *LO = (const double *)a.lo, *HI = (const double *)a.hi, *Y = (const double *)a.y;
    double *X = (double *)a.x, *Sv = (double *)a.s, *MU = (double *)a.mu;
    const double rho1 = sm.rho[0], rho3 = sm.rho[2], rho4 = sm.rho[3];
    const double iq = 1.0 / (double)q;

    double xt[M], xs[M];
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            xt[i] = X[((size_t)i * q + j) * ld + k];
            xs[i] = xt[i];
        }
    const size_t col = (size_t)j * ld + k;
    const double st = Sv[col], yv = Y[col];
    double mu = MU[col];
    if (mu_div != 1.0) mu = mu / mu_div;

#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (i < m) {
            const size_t e = ((size_t)i * a.cq + (size_t)j * a.cj) * ld + k; // coefficient element
            const double a2 = F2[e], a1 = F1[e], b2 = G2[e], b1 = G1[e];
            const int pr = i * q + j;
            const double g0 = cold ? G0[e] : 0.0;
            double others = 0.0;
#pragma unroll
            for (int l = 0; l < M; ++l)
                if (l < m && l != i) others += (a.sweep == ADMM_JACOBI) ? xt[l] : xs[l];
            const double phi = ((st - others) + yv) + mu;
            double C = a2 * iq + 0.5 * rho3, D = a1 * iq - rho3 * phi;
            if (k == 0) {
                C += 0.5 * rho4;
                D -= rho4 * (sm.x1[i] + sm.nu[pr]);
            }
            const double lo = LO[(size_t)i * ld + k], hi = HI[(size_t)i * ld + k];
            double gq_old = 0.0, xn, gq = 0.0;
            // b2 = b1 = 0 (either sign of zero), tested on the integer pipes
            if (((__double_as_longlong(b2) | __double_as_longlong(b1)) << 1) == 0) {
                // no loss on this element (g = beta_0): the terms in beta_2, beta_1
                // vanish and step (a) is the quadratic case of Algorithm 1
                xn = clampd(-D * rcp64(2.0 * C), lo, hi);
            } else {
                gq_old = b2 * xt[i] * xt[i] + b1 * xt[i];
                // u = theta - beta_0 (theta = z + lambda)
                const double u = cold ? -g0 : gq_old + (sm.zeta[pr] + sm.lam[pr]);
                const double A = 0.5 * rho1 * b2 * b2;
                const double B = rho1 * b2 * b1;
                C += 0.5 * rho1 * (b1 * b1 - 2.0 * b2 * u);
                D -= rho1 * b1 * u;
                xn = quartic_min64_seeded(A, B, C, D, lo, hi, a.xmin_mode);
                gq = b2 * xn * xn + b1 * xn;
            }
            xs[i] = xn;
            gs[i] += gq;
            if (check) {
                // z_k - z~_k = D_k + (lambda_new - lambda - zeta); D_k = g(x) - g(x~),
                // or g(x) at the zero start where z~ = 0.
                const double dk = cold ? gq + g0 : gq - gq_old;
                dmx[i] = fmax(dmx[i], dk);
                dmn[i] = fmin(dmn[i], dk);
            }
        }
    }
    double sx = 0.0, dx = 0.0;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            sx += xs[i];
            dx += xs[i] - xt[i];
        }
    const double v = (sx - yv) - mu;
    const double sn = v > 0.0 ? v : 0.0;            // (e)
    const double mun = mu + ((sn - sx) + yv);        // (f)
    if (check) {
        cm_r = fmax(cm_r, fabs((sn - sx) + yv));
        cm_s = fmax(cm_s, fabs((sn - st) - dx));
    }
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) X[((size_t)i * q + j) * ld + k] = xs[i];
    Sv[col] = sn;
    MU[col] = mun;
    if (k == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (i < m) rec[i * 4 + 3] = xs[i];
    }
}

// Warp plan of one pass over the row segments jb..je (at most NWP rows, the
// CTA's warp count) of the chunk [c0, c1): segment s gets warps
// [W_s, W_s+1) with W_s = s + floor((NWP - ns) * (columns before s) /
// (columns in the pass)),
// at least one warp each and the rest in proportion to length, so the
// segments of a CTA run side by side.  The plan depends only on the launch
// shape, so it is the same in every iteration.
struct SegPlan {
    int j;          // row of this warp's segment
    int seg;        // its index within the pass (j - jb)
    int lw, nw;     // this warp's index among the segment's warps, their count
    int64_t s0, s1; // the segment's columns [s0, s1)
};

template <int NWP>
__device__ __forceinline__ SegPlan seg_plan(int64_t c0, int64_t c1, int64_t rs, int jb, int je, int w)
{
    SegPlan p{};
    const int ns = je - jb + 1;
    if (ns == 1) {
        p.j = jb;
        p.lw = w;
        p.nw = NWP;
    } else {
        const int64_t b0 = max(c0, (int64_t)jb * rs), b1 = min(c1, (int64_t)(je + 1) * rs);
        const float scale = (float)(NWP - ns) / (float)(b1 - b0);
        int wlo = 0, whi = NWP;
        for (int t = 0; t < ns; ++t) {
            const int64_t before = max(c0, (int64_t)(jb + t) * rs) - b0;
            const int ws = t + (int)floorf(scale * (float)before);
            if (ws <= w) {
                p.seg = t;
                wlo = ws;
            } else {
                whi = min(whi, ws);
            }
        }
        p.lw = w - wlo;
        p.nw = whi - wlo;
        p.j = jb + p.seg;
    }
    p.s0 = max(c0, (int64_t)p.j * rs);
    p.s1 = min(c1, (int64_t)(p.j + 1) * rs);
    return p;
}

// Rows per pass for the chunk [c0, c1) spanning rows jf..jl: all of them
// side by side (NWP per pass), or one at a time on all warps when that
// takes fewer rounds of column work (long segments, where splitting the
// warps unevenly costs more than the extra reduction barrier, counted as a
// quarter round).  unit: columns per thread and round.
template <int NWP>
__device__ __noinline__ int pass_rows(int64_t c0, int64_t c1, int64_t rs, int jf, int jl, int unit)
{
    const int ns = jl - jf + 1;
    if (ns == 1 || ns > NWP) return NWP;
    int64_t conc = 0, seq4 = (int64_t)(ns - 1); // seq in quarter rounds
    for (int w = 0; w < NWP; ++w) {
        const SegPlan sp = seg_plan<NWP>(c0, c1, rs, jf, jl, w);
        if (sp.lw != 0) continue;
        const int64_t v = (sp.s1 - sp.s0 + unit - 1) / unit;
        conc = max(conc, (v + 32 * sp.nw - 1) / (32 * sp.nw));
        seq4 += 4 * ((v + 32 * NWP - 1) / (32 * NWP));
    }
    return 4 * conc <= seq4 ? NWP : 1;
}

// Columns [c0, c1) of this CTA.
__device__ __forceinline__ void cta_columns(const SingleArgs &a, int unit, int64_t &c0, int64_t &c1)
{
    if (a.pieces > 0) {
        const int j = (int)blockIdx.x / a.pieces, t = (int)blockIdx.x - j * a.pieces;
        c0 = (int64_t)j * a.rs + piece_bound(t, a.rs, a.pieces, unit);
        c1 = (int64_t)j * a.rs + piece_bound(t + 1, a.rs, a.pieces, unit);
    } else {
        c0 = (int64_t)blockIdx.x * a.chunk;
        c1 = min(c0 + a.chunk, a.ncols);
    }
}

// CTAs whose columns touch row j.
__device__ __forceinline__ int row_ctas(const SingleArgs &a, int j)
{
    if (a.pieces > 0) return a.pieces;
    const int64_t rbeg = (int64_t)j * a.rs;
    return (int)((rbeg + a.rs - 1) / a.chunk - rbeg / a.chunk) + 1;
}

// Partial record of row j written by this CTA (position among the CTAs
// touching row j, in column order).
__device__ __forceinline__ double *seg_record(const SingleArgs &a, int par, int j)
{
    const int pos = a.pieces > 0 ? (int)blockIdx.x % a.pieces
                                 : (int)blockIdx.x - (int)(((int64_t)j * a.rs) / a.chunk);
    return a.part + ((size_t)(par * a.q + j) * a.nbmax + pos) * a.m * 4;
}

// Reduction of one pass of row segments into their partial records: warp
// sums by shuffles, then per (segment, source) the sum over that segment's
// warps in warp order.
template <int M, int NWP>
__device__ __forceinline__ void flush_segments(const SingleArgs &a, int par, int jb, const double *gs,
                                               const double *dmx, const double *dmn, bool check, int m,
                                               const SegPlan &sp, const Sm &sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            double v = warp_sum(gs[i]);
            double hi = check ? warp_max(dmx[i]) : 0.0;
            double lo = check ? warp_min(dmn[i]) : 0.0;
            if (lane == 0) {
                sm.red[(w * kMaxM + i) * 3 + 0] = v;
                sm.red[(w * kMaxM + i) * 3 + 1] = hi;
                sm.red[(w * kMaxM + i) * 3 + 2] = lo;
            }
        }
    if (lane == 0) sm.segof[w] = sp.seg;
    __syncthreads();
    if (threadIdx.x < NWP * m) {
        const int sg = threadIdx.x / m, i = threadIdx.x - sg * m;
        double v = 0.0, hi = -INFINITY, lo = INFINITY;
        bool any = false;
        for (int ww = 0; ww < NWP; ++ww)
            if (sm.segof[ww] == sg) {
                any = true;
                v += sm.red[(ww * kMaxM + i) * 3 + 0];
                hi = fmax(hi, sm.red[(ww * kMaxM + i) * 3 + 1]);
                lo = fmin(lo, sm.red[(ww * kMaxM + i) * 3 + 2]);
            }
        if (any) {
            double *rec = seg_record(a, par, jb + sg);
            rec[i * 4 + 0] = v;
            rec[i * 4 + 1] = hi;
            rec[i * 4 + 2] = lo;
        }
    }
    __syncthreads();
}

// Mixed variant, on the FP32 pipes: float-float sums and FP32 max / min in
// a fixed order; only the finished records are converted to FP64.
template <int M, int NWP>
__device__ __forceinline__ void flush_segments32(const SingleArgs &a, int par, int jb, const float2 *ghi,
                                                 const float2 *glo, const float *fmx, const float *fmn, bool check,
                                                 int m, const SegPlan &sp, const Sm &sm)
{
    float *red = (float *)sm.red; // [NWP][kMaxM][4] floats
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            FF v = lanes_sum(ghi[i], glo[i]);
            float hi = fmx[i], lo = fmn[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const FF u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
                v = ff_add(v, u);
                if (check) {
                    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                }
            }
            if (lane == 0) {
                red[(w * kMaxM + i) * 4 + 0] = v.hi;
                red[(w * kMaxM + i) * 4 + 1] = v.lo;
                red[(w * kMaxM + i) * 4 + 2] = hi;
                red[(w * kMaxM + i) * 4 + 3] = lo;
            }
        }
    if (lane == 0) sm.segof[w] = sp.seg;
    __syncthreads();
    if (threadIdx.x < NWP * m) {
        const int sg = threadIdx.x / m, i = threadIdx.x - sg * m;
        FF v = {0.0f, 0.0f};
        float hi = -INFINITY, lo = INFINITY;
        bool any = false;
        for (int ww = 0; ww < NWP; ++ww)
            if (sm.segof[ww] == sg) {
                any = true;
                v = ff_add(v, FF{red[(ww * kMaxM + i) * 4 + 0], red[(ww * kMaxM + i) * 4 + 1]});
                hi = fmaxf(hi, red[(ww * kMaxM + i) * 4 + 2]);
                lo = fminf(lo, red[(ww * kMaxM + i) * 4 + 3]);
            }
        if (any) {
            double *rec = seg_record(a, par, jb + sg);
            rec[i * 4 + 0] = (double)v.hi + (double)v.lo;
            rec[i * 4 + 1] = check ? (double)hi : 0.0;
            rec[i * 4 + 2] = check ? (double)lo : 0.0;
        }
    }
    __syncthreads();
}

// MINB: CTAs per SM the register budget is sized for.  FP64 takes 1 (its
// element update needs about 250 registers); the mixed kernel comes in both:
// 1 for problems that fill at most one CTA per SM (no spills), 2 otherwise.
template <int M, int PREC, int MINB, int NT>
__global__ void __launch_bounds__(NT, MINB) single_kernel(SingleArgs a)
{
    constexpr int NWP = NT / 32;
    extern __shared__ double smem[];
    constexpr bool MIXED = PREC != ADMM_FP64;
    constexpr int VW = kMixedVW;
    const int m = a.m, q = a.q, n = a.n, mq = m * q, rs = a.rs;
    const Sm sm = carve(smem, m, q);
    for (int t = threadIdx.x; t < scal_size(m, q); t += NT) smem[t] = a.scal[t];
    __syncthreads();
    if (MIXED)
        for (int pr = threadIdx.x; pr < mq; pr += NT) {
            sm.uoff[pr] = (float)(sm.zeta[pr] + sm.lam[pr]);
            sm.x1nu[pr] = (float)(sm.x1[pr / q] + sm.nu[pr]);
        }
    __syncthreads();

    int64_t c0, c1;
    cta_columns(a, MIXED ? VW : 1, c0, c1);
    const int jf = (int)(c0 / rs), jl = (int)((c1 - 1) / rs);
    const int prows = pass_rows<NWP>(c0, c1, rs, jf, jl, MIXED ? VW : 1);
    unsigned nbar = 0;
    unsigned esc = 0;
    bool ok = true, conv = false;
    int it;
    double res[7] = {0, 0, 0, 0, 0, 0, 0}; // r1 r2 r3 r4 s1 s2 s3 (unscaled s)
    double r_last = INFINITY, s_last = INFINITY;
    double kappa = sm.rho[1] / (sm.rho[0] + (double)n * sm.rho[1]); // step (b); renewed when rho changes

    for (it = 1; it <= a.max_iter; ++it) {
        const bool check = (it % a.check_every == 0) || (it == a.max_iter);
        const int par = it & 1;
        const bool cold = sm.flags[0] != 0.0;
        const double mu_div = sm.flags[1];
        double cm_r = 0.0, cm_s = 0.0;
        float fcr_all = 0.0f, fcs_all = 0.0f;

        // ---- phase 1: element updates and segment partials --------------
        // The rows j the chunk touches are taken prows at a time; within a
        // pass every row segment gets its own warps, so its segments run
        // concurrently and one reduction barrier closes them all.
        for (int jb = jf; jb <= jl; jb += prows) {
            const SegPlan sp = seg_plan<NWP>(c0, c1, rs, jb, min(jl, jb + prows - 1), threadIdx.x >> 5);
            const int j = sp.j;
            double *rec = seg_record(a, par, j);
            // row-local column range of the segment (k), and this thread's start and step
            const int kb = (int)(sp.s0 - (int64_t)j * rs), ke = (int)(sp.s1 - (int64_t)j * rs);
            const int first = sp.lw * 32 + (threadIdx.x & 31), stride = sp.nw * 32;
            if constexpr (!MIXED) {
                double gs[M], dmx[M], dmn[M];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    gs[i] = 0.0;
                    dmx[i] = -INFINITY;
                    dmn[i] = INFINITY;
                }
                for (int k = kb + first; k < ke; k += stride)
                    column64<M>(a, sm, j, k, check, cold, mu_div, gs, dmx, dmn, cm_r, cm_s, rec);
                flush_segments<M, NWP>(a, par, jb, gs, dmx, dmn, check, m, sp, sm);
            } else {
                float2 ghi[M], glo[M]; // per-lane capacity sums of the column pairs
                float fmx[M], fmn[M];
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    ghi[i] = make_float2(0.0f, 0.0f);
                    glo[i] = make_float2(0.0f, 0.0f);
                    fmx[i] = -INFINITY;
                    fmn[i] = INFINITY;
                }
                const float rho1 = (float)sm.rho[0], rho3 = (float)sm.rho[2], rho4 = (float)sm.rho[3];
                const float iq = 1.0f / (float)q;
                float fcr = 0.0f, fcs = 0.0f;
                const ElemF32 ea = {(const float *)a.f2, (const float *)a.f1, (const float *)a.g2,
                                    (const float *)a.g1, (const float *)a.g0, (const float *)a.lo,
                                    (const float *)a.hi, (const float *)a.y,  (float *)a.x,
                                    (float *)a.s,        (float *)a.mu,       (float *)a.s_lo,
                                    (float *)a.mu_lo,    a.n,                 a.m,
                                    a.q,                 a.ld,                a.sweep,
                                    a.xmin_mode,         a.cq,                a.cj,
                                    a.dbg};
                const int kn = min(ke, n); // padding columns k >= n are skipped
                if constexpr (M <= 4) {
                    // every input through the warp's rolling cp.async stage (each CTA keeps its
                    // columns for the whole launch, so its L1 never holds another SM's lines)
                    float2 *stw = (float2 *)((char *)smem + single_carve_bytes(m, q)) +
                                  (size_t)(threadIdx.x >> 5) * roll_slots<M>() * 32 + (threadIdx.x & 31);
                    const int k00 = kb + first * VW;
                    roll_prologue<M>(ea, j, k00, k00 < kn, stw);
                    for (int k0 = k00; k0 < kn; k0 += stride * VW) {
                        const int k0n = k0 + stride * VW < kn ? k0 + stride * VW : -1;
                        vec32<M, VW, PREC == ADMM_MIXED_FP64CUBIC, STAGE_ROLL>(
                            ea, sm.uoff, sm.x1nu, j, k0, check, cold, (float)mu_div, rho1, rho3, rho4, iq, ghi, glo,
                            fmx, fmn, fcr, fcs, esc, rec, stw, k0n);
                    }
                    cp_async_wait0();
                } else {
                    for (int k0 = kb + first * VW; k0 < kn; k0 += stride * VW) {
                        if constexpr (MINB == 2) // several vectors per thread: fetch the next one into L2
                            if (k0 + stride * VW < kn) prefetch_vec32<M>(ea, j, k0 + stride * VW, cold);
                        vec32<M, VW, PREC == ADMM_MIXED_FP64CUBIC>(ea, sm.uoff, sm.x1nu, j, k0, check, cold,
                                                                   (float)mu_div, rho1, rho3, rho4, iq, ghi, glo,
                                                                   fmx, fmn, fcr, fcs, esc, rec);
                    }
                }
                fcr_all = fmaxf(fcr_all, fcr);
                fcs_all = fmaxf(fcs_all, fcs);
                flush_segments32<M, NWP>(a, par, jb, ghi, glo, fmx, fmn, check, m, sp, sm);
            }
        }
        if (MIXED) {
            cm_r = (double)fcr_all;
            cm_s = (double)fcs_all;
        }
        if (check) {
            double v[2] = {cm_r, cm_s};
            block_max<2, NWP>(v, sm);
            if (threadIdx.x == 0) {
                a.cpart[((size_t)par * a.grid + blockIdx.x) * 4 + 0] = v[0];
                a.cpart[((size_t)par * a.grid + blockIdx.x) * 4 + 1] = v[1];
            }
        }
        ++nbar;
        if (!grid_barrier(a.bar, nbar * (unsigned)a.grid, a.status, a.spin_ns, ADMM_ETIMEOUT)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) sm.flags[1] = 1.0; // the pending mu rescale has been applied

        // ---- phase 2: per-(i, j) scalar steps, redundantly in every CTA ---
        const double rho1 = sm.rho[0], rho2 = sm.rho[1], rho3 = sm.rho[2];
        double r2m = 0.0, r3m = 0.0, s1m = 0.0, s2m = 0.0;
        for (int pr = threadIdx.x; pr < mq; pr += NT) {
            const int i = pr / q, j = pr - i * q;
            const int nb = row_ctas(a, j);
            const double *rec = a.part + ((size_t)(par * q + j) * a.nbmax) * m * 4 + i * 4;
            const int stride = m * 4;
            // records of row j, in CTA order; independent loads, fixed order of the sums
            double S = 0.0, dmx = -INFINITY, dmn = INFINITY;
            // x at k = 0: FP64 in the FP64 kernel, FP32 in the first four bytes of the slot in the mixed ones
            const double x0 = MIXED ? (double)__ldcg((const float *)(rec + 3)) : ldcg(rec + 3);
#pragma unroll 8
            for (int t = 0; t < nb; ++t) {
                S += ldcg(rec + (size_t)t * stride);
                if (check) {
                    dmx = fmax(dmx, ldcg(rec + (size_t)t * stride + 1));
                    dmn = fmin(dmn, ldcg(rec + (size_t)t * stride + 2));
                }
            }
            const double lam = sm.lam[pr], zeta = sm.zeta[pr], hh = sm.h[pr], pp = sm.p[pr];
            const double W = (S + a.sumg0[pr]) - (double)n * lam;     // 1'(g(x) - lambda)
            const double lamn = kappa * ((hh + pp) - W);              // (b) + (g)
            const double Z = W + (double)n * lamn;                    // 1'z
            const double cz = Z - pp;
            const double hn = cz < a.c[i] ? cz : a.c[i];              // (d)
            const double pn = pp + (hn - Z);                          // (i)
            if (check) {
                r2m = max_nonneg(r2m, fabs(lamn - lam));
                r3m = max_nonneg(r3m, fabs(hn - Z));
                const double dl = (lamn - lam) - zeta;
                s1m = max_nonneg(s1m, max_nonneg(fabs(dmx + dl), fabs(dmn + dl)));
                s2m = max_nonneg(s2m, fabs(hn - hh));
            }
            sm.lam[pr] = lamn;
            sm.zeta[pr] = lamn - lam;
            sm.h[pr] = hn;
            sm.p[pr] = pn;
            sm.x0[pr] = x0;
        }
        __syncthreads();
        for (int i = threadIdx.x >> 5; i < m; i += NWP) {        // (c), mean over j: warp i, source i
            const int lane = threadIdx.x & 31;
            double sum = 0.0;
            for (int j = lane; j < q; j += 32) sum += sm.x0[i * q + j] - sm.nu[i * q + j];
            sum = warp_sum(sum);
            if (lane == 0) sm.x1n[i] = sum / (double)q;
        }
        __syncthreads();
        double r4m = 0.0;
        for (int pr = threadIdx.x; pr < mq; pr += NT) {          // (h)
            const int i = pr / q;
            const double x0 = sm.x0[pr], x1n = sm.x1n[i];
            sm.nu[pr] = sm.nu[pr] + (x1n - x0);
            if (check) r4m = max_nonneg(r4m, fabs(x0 - x1n));
        }
        __syncthreads();
        if (threadIdx.x < m) sm.x1[threadIdx.x] = sm.x1n[threadIdx.x];
        if (threadIdx.x == 0) sm.flags[0] = 0.0;
        __syncthreads();

        if (check) {
            double r1 = 0.0, s3 = 0.0;
            for (int b = threadIdx.x; b < a.grid; b += NT) {
                r1 = max_nonneg(r1, ldcg(a.cpart + ((size_t)par * a.grid + b) * 4 + 0));
                s3 = max_nonneg(s3, ldcg(a.cpart + ((size_t)par * a.grid + b) * 4 + 1));
            }
            double v[7] = {r1, r2m, r3m, r4m, s1m, s2m, s3};
            block_max<7, NWP>(v, sm);
#pragma unroll
            for (int t = 0; t < 7; ++t) res[t] = v[t];
            const double r = fmax(fmax(v[0], v[1]), fmax(v[2], v[3]));
            const double sg = fmax(fmax(rho1 * v[4], rho2 * v[5]), rho3 * v[6]);
            r_last = r;
            s_last = sg;
            if (r < a.r_tol && sg < a.s_tol) {
                conv = true;
                break;
            }
            if (a.adapt && it < a.max_iter && it >= a.adapt_start) { // Sec. IV-A, duals rescaled
                const double ratio = r / sg, target = a.adapt_target;
                double f = 1.0;
                if (ratio > 1.2 * target) f = a.tau;
                else if (ratio < 0.8 * target) f = 1.0 / a.tau;
                if (f != 1.0) {
                    for (int pr = threadIdx.x; pr < mq; pr += NT) {
                        sm.lam[pr] /= f;
                        sm.p[pr] /= f;
                        sm.nu[pr] /= f;
                    }
                    __syncthreads();
                    if (threadIdx.x < 4) sm.rho[threadIdx.x] *= f;
                    if (threadIdx.x == 0) sm.flags[1] = f;
                    __syncthreads();
                    kappa = sm.rho[1] / (sm.rho[0] + (double)n * sm.rho[1]);
                }
            }
        }
        if (MIXED) {
            for (int pr = threadIdx.x; pr < mq; pr += NT) {
                sm.uoff[pr] = (float)(sm.zeta[pr] + sm.lam[pr]);
                sm.x1nu[pr] = (float)(sm.x1[pr / q] + sm.nu[pr]);
            }
            __syncthreads();
        }
    }
    const int iters = it > a.max_iter ? a.max_iter : it;

    // ---- objective (1/q) sum f(x) of eq. (2): one more barrier -----------
    if (ok) {
        double acc = 0.0;
        for (int64_t cc = c0 + threadIdx.x; cc < c1; cc += NT) {
            const int j = (int)(cc / rs), k = (int)(cc - (int64_t)j * rs);
            if (k >= n) continue;
            for (int i = 0; i < m; ++i) {
                const size_t e = ((size_t)i * q + j) * a.ld + k;
                const size_t ec = ((size_t)i * a.cq + (size_t)j * a.cj) * a.ld + k; // coefficient element
                double f2, f1, f0, x;
                if constexpr (MIXED) {
                    f2 = ((const float *)a.f2)[ec];
                    f1 = ((const float *)a.f1)[ec];
                    f0 = ((const float *)a.f0)[ec];
                    x = ((const float *)a.x)[e];
                } else {
                    f2 = ((const double *)a.f2)[ec];
                    f1 = ((const double *)a.f1)[ec];
                    f0 = ((const double *)a.f0)[ec];
                    x = ((const double *)a.x)[e];
                }
                acc += f2 * x * x + f1 * x + f0;
            }
        }
        acc = warp_sum(acc);
        double escd = warp_sum((double)esc);
        if ((threadIdx.x & 31) == 0) {
            sm.mx[(threadIdx.x >> 5) * 8] = acc;
            sm.mx[(threadIdx.x >> 5) * 8 + 1] = escd;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0, te = 0.0;
            for (int w = 0; w < NWP; ++w) {
                t += sm.mx[w * 8];
                te += sm.mx[w * 8 + 1];
            }
            a.cpart[(size_t)blockIdx.x * 4 + 2] = t;
            a.cpart[(size_t)blockIdx.x * 4 + 3] = te;
        }
        ++nbar;
        ok = grid_barrier(a.bar, nbar * (unsigned)a.grid, a.status, a.spin_ns, ADMM_ETIMEOUT);
    }
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < scal_size(m, q); t += NT) a.scal[t] = smem[t];
        if (threadIdx.x == 0) {
            double obj = 0.0, escs = 0.0;
            if (ok)
                for (int b = 0; b < a.grid; ++b) {
                    obj += ldcg(a.cpart + (size_t)b * 4 + 2);
                    escs += ldcg(a.cpart + (size_t)b * 4 + 3);
                }
            a.info[0] = iters;
            a.info[1] = conv ? 1.0 : 0.0;
            a.info[2] = r_last;
            a.info[3] = s_last;
            for (int t = 0; t < 4; ++t) a.info[4 + t] = res[t];
            for (int t = 0; t < 3; ++t) a.info[8 + t] = res[4 + t] * sm.rho[t];
            a.info[11] = obj / (double)q;
            a.info[12] = ok ? 0.0 : (double)ld_volatile_i32(a.status);
            a.info[13] = escs;
        }
    }
}

template <int M> void *single_fn(int precision, int minb)
{
    switch (precision) {
    case ADMM_MIXED:
        return minb == 1 ? (void *)single_kernel<M, ADMM_MIXED, 1, kBlock>
                         : (void *)single_kernel<M, ADMM_MIXED, 2, kBlock>;
    case ADMM_MIXED_FP64CUBIC:
        return minb == 1 ? (void *)single_kernel<M, ADMM_MIXED_FP64CUBIC, 1, kBlock>
                         : (void *)single_kernel<M, ADMM_MIXED_FP64CUBIC, 2, kBlock>;
    default: return (void *)single_kernel<M, ADMM_FP64, 1, kBlockF64>;
    }
}

void *pick(int precision, int m, int minb)
{
    switch (single_mbound(m)) {
    case 2: return single_fn<2>(precision, minb);
    case 4: return single_fn<4>(precision, minb);
    default: return single_fn<8>(precision, minb);
    }
}

} // namespace

int single_mbound(int m) { return m <= 2 ? 2 : (m <= 4 ? 4 : 8); }

// FP64: 12 warps (one CTA per SM, up to 168 registers a thread); the FP64
// units are shared by the SM, so more warps hide more of their latency.
int single_threads(int precision) { return precision == ADMM_FP64 ? kBlockF64 : kBlock; }

size_t single_smem_bytes(int m, int q, int precision)
{
    const int mb = single_mbound(m);
    size_t stage = 0; // the rolling stage of the mixed kernels, one per warp
    if (precision != ADMM_FP64 && mb <= 4)
        stage = (size_t)(kBlock / 32) * (mb == 2 ? roll_slots<2>() : roll_slots<4>()) * 32 * sizeof(float2);
    return single_carve_bytes(m, q) + stage;
}

int single_blocks_per_sm(int precision, int m, int minb, size_t smem)
{
    void *fn = pick(precision, m, minb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, single_threads(precision), smem) != cudaSuccess)
        return 0;
    return nb;
}

SingleShape single_shape(int precision, int m, int q, int64_t rs, int nsm, size_t smem)
{
    SingleShape sh{};
    const bool mixed = precision != ADMM_FP64;
    const int64_t unit = mixed ? kMixedVW : 1;   // mixed: vectors of kMixedVW columns
    const int64_t ncols = (int64_t)q * rs;
    // Contiguous equal column chunks over as many SMs as there are warps of
    // work (FP64 throughput per SM is the scarce resource), one CTA per SM
    // while that covers every column vector in a single pass, two otherwise.
    sh.minb = (mixed && ncols > (int64_t)nsm * single_threads(precision) * unit) ? 2 : 1;
    int per_sm = single_blocks_per_sm(precision, m, sh.minb, smem);
    if (per_sm < 1 && sh.minb == 2) {
        sh.minb = 1;
        per_sm = single_blocks_per_sm(precision, m, 1, smem);
    }
    if (per_sm < 1) return sh;
    const int64_t g = std::min<int64_t>((int64_t)nsm * per_sm, std::max<int64_t>(1, ncols / (32 * unit)));
    sh.chunk = ((ncols + g - 1) / g + unit - 1) / unit * unit;
    // Row-aligned split when every row gets whole pieces and the largest
    // piece is within 5 % of the flat chunk: no CTA then straddles two rows
    // (a straddling CTA reduces two segments and finishes last).
    const int p = (int)(g / q);
    if (p >= 1) {
        int64_t big = 0;
        for (int t = 0; t < p; ++t)
            big = std::max(big, piece_bound(t + 1, rs, p, (int)unit) - piece_bound(t, rs, p, (int)unit));
        if (piece_bound(1, rs, p, (int)unit) > 0 && 20 * big <= 21 * sh.chunk) {
            sh.pieces = p;
            sh.grid = q * p;
            sh.nbmax = p;
            return sh;
        }
    }
    sh.pieces = 0;
    sh.grid = (int)((ncols + sh.chunk - 1) / sh.chunk);
    sh.nbmax = 1;
    for (int j = 0; j < q; ++j) {
        const int64_t r0 = (int64_t)j * rs, r1 = r0 + rs - 1;
        sh.nbmax = std::max(sh.nbmax, (int)(r1 / sh.chunk - r0 / sh.chunk + 1));
    }
    return sh;
}

cudaError_t launch_single(int precision, int minb, const SingleArgs &a, size_t smem, cudaStream_t st)
{
    void *fn = pick(precision, a.m, minb);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SingleArgs copy = a;
    void *args[] = {(void *)&copy};
    return cudaLaunchCooperativeKernel(fn, dim3(a.grid), dim3(single_threads(precision)), args, smem, st);
}

} // namespace admm_impl

namespace admm_impl {
namespace {
template <class S, class D>
__global__ void convert_rows_kernel(D *dst, int64_t dld, const S *src, int64_t sld, int n, int64_t rows)
{
    const int64_t total = rows * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n;
        const int k = (int)(t - r * n);
        dst[r * dld + k] = (D)src[r * sld + k];
    }
}
int conv_grid(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (total + 255) / 256)); }
} // namespace

void convert_rows_f32_to_f64(double *dst, int64_t dld, const float *src, int64_t sld, int n, int64_t rows,
                             cudaStream_t st)
{
    convert_rows_kernel<float, double><<<conv_grid(rows * n), 256, 0, st>>>(dst, dld, src, sld, n, rows);
}
namespace {
__global__ void ff_to_f64_kernel(double *dst, int64_t dld, const float *hi, const float *lo, int64_t sld, int n,
                                 int64_t rows)
{
    const int64_t total = rows * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n;
        const int k = (int)(t - r * n);
        dst[r * dld + k] = (double)hi[r * sld + k] + (double)lo[r * sld + k];
    }
}
__global__ void f64_to_ff_kernel(float *hi, float *lo, int64_t dld, const double *src, int64_t sld, int n,
                                 int64_t rows)
{
    const int64_t total = rows * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n;
        const int k = (int)(t - r * n);
        const double v = src[r * sld + k];
        const float h = (float)v;
        hi[r * dld + k] = h;
        lo[r * dld + k] = (float)(v - (double)h);
    }
}
} // namespace

void convert_rows_ff_to_f64(double *dst, int64_t dld, const float *hi, const float *lo, int64_t sld, int n,
                            int64_t rows, cudaStream_t st)
{
    ff_to_f64_kernel<<<conv_grid(rows * n), 256, 0, st>>>(dst, dld, hi, lo, sld, n, rows);
}
void split_rows_f64_to_ff(float *hi, float *lo, int64_t dld, const double *src, int64_t sld, int n, int64_t rows,
                          cudaStream_t st)
{
    f64_to_ff_kernel<<<conv_grid(rows * n), 256, 0, st>>>(hi, lo, dld, src, sld, n, rows);
}

void convert_rows_f64_to_f32(float *dst, int64_t dld, const double *src, int64_t sld, int n, int64_t rows,
                             cudaStream_t st)
{
    convert_rows_kernel<double, float><<<conv_grid(rows * n), 256, 0, st>>>(dst, dld, src, sld, n, rows);
}
} // namespace admm_impl

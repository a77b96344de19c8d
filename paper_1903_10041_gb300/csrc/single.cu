// Persistent single-instance solve kernel: the whole ADMM loop of App. A on
// the device, one cooperative launch per solve.
//
// Work split.  The q*n columns (j, k) are taken in j-major order and cut
// into `grid` contiguous chunks of `chunk` columns, one per CTA, so every
// CTA does the same number of element updates.  The thread that owns a
// column updates all m sources of it in registers (step (a) sweeps the
// sources in order, so the Gauss-Seidel sums over l != i stay local), then
// steps (e) and (f) for that column.  The per-(i, j) sums over k that steps
// (b) and (d) and the residuals need are segmented reductions: each CTA
// reduces each row segment it owns (warp shuffles, then shared memory) into
// a partial record; after one grid barrier every CTA adds the records of
// each row in a fixed order and runs the per-(i, j) scalar steps (b), (c),
// (d), (g), (h), (i), the residuals and the stop test redundantly, so all
// CTAs hold identical scalars and take the same stop decision without a
// second barrier.  Partial records are double-buffered by iteration parity.
//
// Identities used (derived from steps (b) and (g)): after every iteration
// lambda^(i,j) is constant over k and z_k = g_k(x_k) + zeta with
// zeta = lambda_new - lambda_old, so theta_k = z_k + lambda =
// g_k(x~_k) + zeta + lambda needs no per-element z or lambda.  The zero start
// (z = 0, the paper's iteration from zeros) is flagged `cold`, where
// theta = 0 instead.
#include "common.cuh"
#include "internal.h"
#include "quartic64.cuh"

namespace admm_impl {

namespace {

struct Sm {
    double *lam, *zeta, *h, *p, *nu, *x1, *rho, *flags; // mirror of the scalar state
    double *x0;   // [mq]
    double *x1n;  // [kMaxM]
    double *red;  // [kWarps][kMaxM][3]
    double *mx;   // [kWarps][8]
    double *bc;   // [16] broadcast
};

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
    t += kWarps * kMaxM * 3;
    s.mx = t;
    t += kWarps * 8;
    s.bc = t;
    return s;
}

// Block-wide max of up to 8 values; every thread gets the results in out[].
template <int NV> __device__ __forceinline__ void block_max(double *v, const Sm &sm)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        double r = warp_max(v[t]);
        if (lane == 0) sm.mx[w * 8 + t] = r;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double r = 0.0;
        for (int ww = 0; ww < kWarps; ++ww) r = fmax(r, sm.mx[ww * 8 + threadIdx.x]);
        sm.bc[threadIdx.x] = r;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = sm.bc[t];
    __syncthreads();
}

// Step (a) for all sources of column (j, k), then (e), (f) for the column.
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
            const size_t e = ((size_t)i * q + j) * ld + k;
            const double a2 = F2[e], a1 = F1[e], b2 = G2[e], b1 = G1[e];
            const int pr = i * q + j;
            const double gq_old = b2 * xt[i] * xt[i] + b1 * xt[i];
            const double g0 = cold ? G0[e] : 0.0;
            // u = theta - beta_0 (theta = z + lambda)
            const double u = cold ? -g0 : gq_old + (sm.zeta[pr] + sm.lam[pr]);
            double others = 0.0;
#pragma unroll
            for (int l = 0; l < M; ++l)
                if (l < m && l != i) others += (a.sweep == ADMM_JACOBI) ? xt[l] : xs[l];
            const double phi = ((st - others) + yv) + mu;
            const double A = 0.5 * rho1 * b2 * b2;
            const double B = rho1 * b2 * b1;
            double C = a2 * iq + 0.5 * rho1 * (b1 * b1 - 2.0 * b2 * u) + 0.5 * rho3;
            double D = a1 * iq - rho1 * b1 * u - rho3 * phi;
            if (k == 0) {
                C += 0.5 * rho4;
                D -= rho4 * (sm.x1[i] + sm.nu[pr]);
            }
            const double xn = quartic_min64(A, B, C, D, LO[(size_t)i * ld + k], HI[(size_t)i * ld + k],
                                            a.xmin_mode);
            xs[i] = xn;
            const double gq = b2 * xn * xn + b1 * xn;
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

template <int M>
__device__ __forceinline__ void flush_segment(double *rec, double *gs, double *dmx, double *dmn, bool check,
                                              int m, const Sm &sm)
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
    __syncthreads();
    if (threadIdx.x < m) {
        const int i = threadIdx.x;
        double v = 0.0, hi = -INFINITY, lo = INFINITY;
        for (int ww = 0; ww < kWarps; ++ww) {
            v += sm.red[(ww * kMaxM + i) * 3 + 0];
            hi = fmax(hi, sm.red[(ww * kMaxM + i) * 3 + 1]);
            lo = fmin(lo, sm.red[(ww * kMaxM + i) * 3 + 2]);
        }
        rec[i * 4 + 0] = v;
        rec[i * 4 + 1] = hi;
        rec[i * 4 + 2] = lo;
    }
    __syncthreads();
}

template <int M> __global__ void __launch_bounds__(kBlock, 1) single_fp64_kernel(SingleArgs a)
{
    extern __shared__ double smem[];
    const int m = a.m, q = a.q, n = a.n, mq = m * q;
    const Sm sm = carve(smem, m, q);
    for (int t = threadIdx.x; t < scal_size(m, q); t += kBlock) smem[t] = a.scal[t];
    __syncthreads();

    const int64_t c0 = (int64_t)blockIdx.x * a.chunk;
    const int64_t c1 = min(c0 + a.chunk, a.ncols);
    const int jf = (int)(c0 / n), jl = (int)((c1 - 1) / n);
    unsigned nbar = 0;
    bool ok = true, conv = false;
    int it;
    double res[7] = {0, 0, 0, 0, 0, 0, 0}; // r1 r2 r3 r4 s1 s2 s3 (unscaled s)
    double r_last = INFINITY, s_last = INFINITY;

    for (it = 1; it <= a.max_iter; ++it) {
        const bool check = (it % a.check_every == 0) || (it == a.max_iter);
        const int par = it & 1;
        const bool cold = sm.flags[0] != 0.0;
        const double mu_div = sm.flags[1];
        double cm_r = 0.0, cm_s = 0.0;

        // ---- phase 1: element updates and segment partials --------------
        for (int j = jf; j <= jl; ++j) {
            const int64_t s0 = max(c0, (int64_t)j * n), s1 = min(c1, (int64_t)(j + 1) * n);
            double gs[M], dmx[M], dmn[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                gs[i] = 0.0;
                dmx[i] = -INFINITY;
                dmn[i] = INFINITY;
            }
            double *rec = a.part + ((size_t)(par * a.grid + blockIdx.x) * a.slots + (j - jf)) * m * 4;
            for (int64_t cc = s0 + threadIdx.x; cc < s1; cc += kBlock)
                column64<M>(a, sm, j, (int)(cc - (int64_t)j * n), check, cold, mu_div, gs, dmx, dmn, cm_r,
                            cm_s, rec);
            flush_segment<M>(rec, gs, dmx, dmn, check, m, sm);
        }
        if (check) {
            double v[2] = {cm_r, cm_s};
            block_max<2>(v, sm);
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
        const double kappa = rho2 / (rho1 + (double)n * rho2);
        double r2m = 0.0, r3m = 0.0, s1m = 0.0, s2m = 0.0;
        for (int pr = threadIdx.x; pr < mq; pr += kBlock) {
            const int i = pr / q, j = pr - i * q;
            const int64_t rs = (int64_t)j * n;
            const int b0 = (int)(rs / a.chunk), b1 = (int)((rs + n - 1) / a.chunk);
            double S = 0.0, dmx = -INFINITY, dmn = INFINITY, x0 = 0.0;
            for (int b = b0; b <= b1; ++b) {
                const int slot = j - (int)(((int64_t)b * a.chunk) / n);
                const double *rec = a.part + ((size_t)(par * a.grid + b) * a.slots + slot) * m * 4 + i * 4;
                S += ldcg(rec);
                if (check) {
                    dmx = fmax(dmx, ldcg(rec + 1));
                    dmn = fmin(dmn, ldcg(rec + 2));
                }
                if (b == b0) x0 = ldcg(rec + 3);
            }
            const double lam = sm.lam[pr], zeta = sm.zeta[pr], hh = sm.h[pr], pp = sm.p[pr];
            const double W = (S + a.sumg0[pr]) - (double)n * lam;     // 1'(g(x) - lambda)
            const double lamn = kappa * ((hh + pp) - W);              // (b) + (g)
            const double Z = W + (double)n * lamn;                    // 1'z
            const double cz = Z - pp;
            const double hn = cz < a.c[i] ? cz : a.c[i];              // (d)
            const double pn = pp + (hn - Z);                          // (i)
            if (check) {
                r2m = fmax(r2m, fabs(lamn - lam));
                r3m = fmax(r3m, fabs(hn - Z));
                const double dl = (lamn - lam) - zeta;
                s1m = fmax(s1m, fmax(fabs(dmx + dl), fabs(dmn + dl)));
                s2m = fmax(s2m, fabs(hn - hh));
            }
            sm.lam[pr] = lamn;
            sm.zeta[pr] = lamn - lam;
            sm.h[pr] = hn;
            sm.p[pr] = pn;
            sm.x0[pr] = x0;
        }
        __syncthreads();
        if (threadIdx.x < m) {                                       // (c), mean over j
            const int i = threadIdx.x;
            double sum = 0.0;
            for (int j = 0; j < q; ++j) sum += sm.x0[i * q + j] - sm.nu[i * q + j];
            sm.x1n[i] = sum / (double)q;
        }
        __syncthreads();
        double r4m = 0.0;
        for (int pr = threadIdx.x; pr < mq; pr += kBlock) {          // (h)
            const int i = pr / q;
            const double x0 = sm.x0[pr], x1n = sm.x1n[i];
            sm.nu[pr] = sm.nu[pr] + (x1n - x0);
            if (check) r4m = fmax(r4m, fabs(x0 - x1n));
        }
        __syncthreads();
        if (threadIdx.x < m) sm.x1[threadIdx.x] = sm.x1n[threadIdx.x];
        if (threadIdx.x == 0) sm.flags[0] = 0.0;
        __syncthreads();

        if (check) {
            double r1 = 0.0, s3 = 0.0;
            for (int b = threadIdx.x; b < a.grid; b += kBlock) {
                r1 = fmax(r1, ldcg(a.cpart + ((size_t)par * a.grid + b) * 4 + 0));
                s3 = fmax(s3, ldcg(a.cpart + ((size_t)par * a.grid + b) * 4 + 1));
            }
            double v[7] = {r1, r2m, r3m, r4m, s1m, s2m, s3};
            block_max<7>(v, sm);
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
            if (a.adapt && it < a.max_iter) { // Sec. IV-A, duals rescaled by rho_old / rho_new
                const double ratio = r / sg, target = a.r_tol / a.s_tol;
                double f = 1.0;
                if (ratio > 1.2 * target) f = a.tau;
                else if (ratio < 0.8 * target) f = 1.0 / a.tau;
                if (f != 1.0) {
                    for (int pr = threadIdx.x; pr < mq; pr += kBlock) {
                        sm.lam[pr] /= f;
                        sm.p[pr] /= f;
                        sm.nu[pr] /= f;
                    }
                    __syncthreads();
                    if (threadIdx.x < 4) sm.rho[threadIdx.x] *= f;
                    if (threadIdx.x == 0) sm.flags[1] = f;
                    __syncthreads();
                }
            }
        }
    }
    const int iters = it > a.max_iter ? a.max_iter : it;

    // ---- objective (1/q) sum f(x) of eq. (2): one more barrier -----------
    if (ok) {
        const double *F2 = (const double *)a.f2, *F1 = (const double *)a.f1, *F0 = (const double *)a.f0;
        const double *X = (const double *)a.x;
        double acc = 0.0;
        for (int64_t cc = c0 + threadIdx.x; cc < c1; cc += kBlock) {
            const int j = (int)(cc / n), k = (int)(cc - (int64_t)j * n);
            for (int i = 0; i < m; ++i) {
                const size_t e = ((size_t)i * q + j) * a.ld + k;
                acc += F2[e] * X[e] * X[e] + F1[e] * X[e] + F0[e];
            }
        }
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) sm.mx[(threadIdx.x >> 5) * 8] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += sm.mx[w * 8];
            a.cpart[(size_t)blockIdx.x * 4 + 2] = t;
        }
        ++nbar;
        ok = grid_barrier(a.bar, nbar * (unsigned)a.grid, a.status, a.spin_ns, ADMM_ETIMEOUT);
    }
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < scal_size(m, q); t += kBlock) a.scal[t] = smem[t];
        if (threadIdx.x == 0) {
            double obj = 0.0;
            if (ok)
                for (int b = 0; b < a.grid; ++b) obj += ldcg(a.cpart + (size_t)b * 4 + 2);
            a.info[0] = iters;
            a.info[1] = conv ? 1.0 : 0.0;
            a.info[2] = r_last;
            a.info[3] = s_last;
            for (int t = 0; t < 4; ++t) a.info[4 + t] = res[t];
            for (int t = 0; t < 3; ++t) a.info[8 + t] = res[4 + t] * sm.rho[t];
            a.info[11] = obj / (double)q;
            a.info[12] = ok ? 0.0 : (double)ld_volatile_i32(a.status);
        }
    }
}

template <int M> void *single_fn(int precision)
{
    (void)precision;
    return (void *)single_fp64_kernel<M>;
}

void *pick(int precision, int m)
{
    switch (single_mbound(m)) {
    case 2: return single_fn<2>(precision);
    case 4: return single_fn<4>(precision);
    default: return single_fn<8>(precision);
    }
}

} // namespace

int single_mbound(int m) { return m <= 2 ? 2 : (m <= 4 ? 4 : 8); }

size_t single_smem_bytes(int m, int q)
{
    const int mq = m * q;
    return sizeof(double) * ((size_t)scal_size(m, q) + mq + kMaxM + kWarps * kMaxM * 3 + kWarps * 8 + 16);
}

int single_blocks_per_sm(int precision, int m, size_t smem)
{
    void *fn = pick(precision, m);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBlock, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_single(int precision, const SingleArgs &a, size_t smem, cudaStream_t st)
{
    void *fn = pick(precision, a.m);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SingleArgs copy = a;
    void *args[] = {(void *)&copy};
    return cudaLaunchCooperativeKernel(fn, dim3(a.grid), dim3(kBlock), args, smem, st);
}

} // namespace admm_impl

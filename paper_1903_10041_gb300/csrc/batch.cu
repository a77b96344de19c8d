// Batched solve: thousands of independent instances of uneven n, m, q in one
// persistent launch (mixed precision).
//
// Each instance is solved by one team of threads that runs the whole ADMM
// loop of App. A for it with team-local synchronisation only: a whole CTA
// for large instances, or a single warp for small ones (so a CTA of W warps
// holds W small instances at once).  Teams take work from two global
// queues of instance ids, large ones first, each sorted by decreasing
// estimated work (longest-processing-time order), so a CTA that finishes
// early takes the next instance.  Each instance stops on its own stop test.
//
// The largest instances are solved by a thread-block cluster (2-8 CTAs on
// neighbouring SMs): each CTA reduces its part of every row into records in
// its own shared memory, one hardware cluster barrier per iteration follows,
// and every CTA reads all CTAs' records through distributed shared memory in
// rank order and runs the scalar steps redundantly.
//
// Per iteration a team sweeps the rows j = 1..q of its instance; within a
// row its threads take consecutive column vectors (coalesced) and run the
// element update of mixed_elem.cuh; the row's sums over k are reduced
// across the team in a fixed order into a record in shared memory, and the
// per-(i, j) scalar steps, residuals and stop test follow on the team.  The
// arithmetic and its order depend only on the instance's own shape and its
// team kind (fixed by the instance's size), so an instance gives the same
// bits alone and in any mix.
//
// An iteration budget lets a launch stop every instance after a given
// number of iterations with its state saved; the serving loop uses it to
// run the batch in ticks and admit new instances between ticks.
#include <algorithm>

#include <cooperative_groups.h>

#include "batch.h"
#include "common.cuh"
#include "mixed_elem.cuh"

namespace admm_impl {

namespace {

// Team of NT threads (32 = one warp; or the whole CTA).
template <int NT> struct Team {
    int tid;
    __device__ __forceinline__ void sync() const
    {
        if constexpr (NT == 32) __syncwarp();
        else __syncthreads();
    }
};

// Team-wide float-float sum and FP32 max/min for m row records.
template <int NT, int M>
__device__ __forceinline__ void team_flush(const Team<NT> &T, double *rec, const float *ghi, const float *glo,
                                           const float *fmx, const float *fmn, bool check, int m, float *red)
{
    const int lane = T.tid & 31, w = T.tid >> 5;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (i < m) {
            FF v = ff_norm(ghi[i], glo[i]);
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
            if (NT == 32) {
                if (lane == 0) {
                    rec[i * 4 + 0] = (double)v.hi + (double)v.lo;
                    rec[i * 4 + 1] = check ? (double)hi : 0.0;
                    rec[i * 4 + 2] = check ? (double)lo : 0.0;
                }
            } else if (lane == 0) {
                red[(w * kMaxM + i) * 4 + 0] = v.hi;
                red[(w * kMaxM + i) * 4 + 1] = v.lo;
                red[(w * kMaxM + i) * 4 + 2] = hi;
                red[(w * kMaxM + i) * 4 + 3] = lo;
            }
        }
    if constexpr (NT > 32) {
        __syncthreads();
        if (T.tid < m) {
            const int i = T.tid;
            FF v = {0.0f, 0.0f};
            float hi = -INFINITY, lo = INFINITY;
            for (int ww = 0; ww < NT / 32; ++ww) {
                v = ff_add(v, FF{red[(ww * kMaxM + i) * 4 + 0], red[(ww * kMaxM + i) * 4 + 1]});
                hi = fmaxf(hi, red[(ww * kMaxM + i) * 4 + 2]);
                lo = fminf(lo, red[(ww * kMaxM + i) * 4 + 3]);
            }
            rec[i * 4 + 0] = (double)v.hi + (double)v.lo;
            rec[i * 4 + 1] = check ? (double)hi : 0.0;
            rec[i * 4 + 2] = check ? (double)lo : 0.0;
        }
    }
    T.sync();
}

// Team-wide max of NV doubles (every thread gets the result).
template <int NT, int NV> __device__ __forceinline__ void team_max(const Team<NT> &T, double *v, double *scr)
{
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = warp_max(v[t]);
    if constexpr (NT > 32) {
        const int lane = T.tid & 31, w = T.tid >> 5;
        if (lane == 0)
            for (int t = 0; t < NV; ++t) scr[w * 8 + t] = v[t];
        __syncthreads();
        for (int t = 0; t < NV; ++t) {
            double r = 0.0;
            for (int ww = 0; ww < NT / 32; ++ww) r = fmax(r, scr[ww * 8 + t]);
            v[t] = r;
        }
        __syncthreads();
    }
}

// Team-wide FP64 sum (fixed order), every thread gets the result.
template <int NT> __device__ __forceinline__ double team_sum(const Team<NT> &T, double v, double *scr)
{
    v = warp_sum(v);
    if constexpr (NT > 32) {
        const int lane = T.tid & 31, w = T.tid >> 5;
        if (lane == 0) scr[w * 8] = v;
        __syncthreads();
        double r = 0.0;
        for (int ww = 0; ww < NT / 32; ++ww) r += scr[ww * 8];
        __syncthreads();
        return r;
    }
    return v;
}

template <int NT, int M>
__device__ void solve_instance(const BatchArgs &a, int id, double *slice, int tid)
{
    const Team<NT> T{tid};
    const BatchInst I = a.inst[id];
    const int n = I.n, m = I.m, q = I.q, mq = m * q;
    constexpr int VW = kMixedVW;

    // team slice: scalar state | row records [q][m][4] | x1n | scratch | red (floats) | uoff (floats)
    double *scal = slice;
    double *lam = scal, *zeta = scal + mq, *hh = scal + 2 * mq, *pp = scal + 3 * mq, *nu = scal + 4 * mq;
    double *x1 = scal + 5 * mq, *rho = x1 + m, *flags = rho + 4;
    double *recs = slice + scal_size(m, q);
    double *x1n = recs + (size_t)q * m * 4;
    double *scr = x1n + kMaxM;
    float *red = (float *)(scr + kWarpsMax * 8);
    float *uoff = red + kWarpsMax * kMaxM * 4;

    double *gscal = a.scal + I.off_scal;
    double *out = a.out + (size_t)id * kInfo;
    if (out[14] != 0.0) return; // already finished (converged or out of iterations)
    for (int t = tid; t < scal_size(m, q); t += NT) scal[t] = gscal[t];
    T.sync();
    for (int pr = tid; pr < mq; pr += NT) uoff[pr] = (float)(zeta[pr] + lam[pr]);
    const int it0 = (int)out[0];
    T.sync();

    const ElemF32 ea = {a.f2 + I.off_e, a.f1 + I.off_e, a.g2 + I.off_e, a.g1 + I.off_e, a.g0 + I.off_e,
                        a.lo + I.off_b, a.hi + I.off_b, a.y + I.off_c,  a.x + I.off_e,  a.s + I.off_c,
                        a.mu + I.off_c, a.s_lo + I.off_c, a.mu_lo + I.off_c, n, m, q, I.ld, a.sweep, a.xmin_mode};
    const double *cc = a.c + I.off_src;
    const double *sumg0 = a.sumg0 + I.off_pair;
    const int nv = (n + VW - 1) / VW;
    unsigned esc = 0;
    bool conv = false;
    double res[7] = {out[4], out[5], out[6], out[7], out[8], out[9], out[10]};
    double r_last = out[2], s_last = out[3];
    int it = it0;
    const int it_end = a.iter_budget > 0 ? min(a.max_iter, it0 + a.iter_budget) : a.max_iter;

    while (it < it_end) {
        ++it;
        const bool check = (it % a.check_every == 0) || (it == a.max_iter);
        const bool cold = flags[0] != 0.0;
        const float mu_div = (float)flags[1];
        const float rho1 = (float)rho[0], rho3 = (float)rho[2], rho4 = (float)rho[3];
        const float iq = 1.0f / (float)q;
        float fcr = 0.0f, fcs = 0.0f;
        for (int j = 0; j < q; ++j) {
            float ghi[M], glo[M], fmx[M], fmn[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                ghi[i] = 0.0f;
                glo[i] = 0.0f;
                fmx[i] = -INFINITY;
                fmn[i] = INFINITY;
            }
            double *rec = recs + (size_t)j * m * 4;
            for (int v = tid; v < nv; v += NT)
                vec32<M, VW, false>(ea, uoff, x1, nu, j, v * VW, check, cold, mu_div, rho1, rho3, rho4, iq, ghi, glo,
                                    fmx, fmn, fcr, fcs, esc, rec);
            team_flush<NT, M>(T, rec, ghi, glo, fmx, fmn, check, m, red);
        }
        if (tid == 0) flags[1] = 1.0;

        // per-(i, j) scalar steps, as in the single-instance kernel
        const double r1 = rho[0], r2 = rho[1], r3 = rho[2];
        const double kappa = r2 / (r1 + (double)n * r2);
        double r2m = 0.0, r3m = 0.0, s1m = 0.0, s2m = 0.0;
        for (int pr = tid; pr < mq; pr += NT) {
            const int i = pr / q, j = pr - i * q;
            const double *rec = recs + ((size_t)j * m + i) * 4;
            const double S = rec[0], dmx = rec[1], dmn = rec[2], x0 = rec[3];
            const double lm = lam[pr], zt = zeta[pr], h0 = hh[pr], p0 = pp[pr];
            const double W = (S + sumg0[pr]) - (double)n * lm;
            const double lamn = kappa * ((h0 + p0) - W);
            const double Z = W + (double)n * lamn;
            const double cz = Z - p0;
            const double hn = cz < cc[i] ? cz : cc[i];
            const double pn = p0 + (hn - Z);
            if (check) {
                r2m = fmax(r2m, fabs(lamn - lm));
                r3m = fmax(r3m, fabs(hn - Z));
                const double dl = (lamn - lm) - zt;
                s1m = fmax(s1m, fmax(fabs(dmx + dl), fabs(dmn + dl)));
                s2m = fmax(s2m, fabs(hn - h0));
            }
            lam[pr] = lamn;
            zeta[pr] = lamn - lm;
            hh[pr] = hn;
            pp[pr] = pn;
        }
        T.sync();
        if (tid < m) {
            const int i = tid;
            double sum = 0.0;
            for (int j = 0; j < q; ++j) sum += recs[((size_t)j * m + i) * 4 + 3] - nu[i * q + j];
            x1n[i] = sum / (double)q;
        }
        T.sync();
        double r4m = 0.0;
        for (int pr = tid; pr < mq; pr += NT) {
            const int i = pr / q, j = pr - i * q;
            const double x0 = recs[((size_t)j * m + i) * 4 + 3], xn = x1n[i];
            nu[pr] = nu[pr] + (xn - x0);
            if (check) r4m = fmax(r4m, fabs(x0 - xn));
        }
        T.sync();
        if (tid < m) x1[tid] = x1n[tid];
        if (tid == 0) flags[0] = 0.0;
        T.sync();
        if (check) {
            double v[7] = {(double)fcr, r2m, r3m, r4m, s1m, s2m, (double)fcs};
            team_max<NT, 7>(T, v, scr);
#pragma unroll
            for (int t = 0; t < 7; ++t) res[t] = v[t];
            const double r = fmax(fmax(v[0], v[1]), fmax(v[2], v[3]));
            const double sg = fmax(fmax(r1 * v[4], r2 * v[5]), r3 * v[6]);
            r_last = r;
            s_last = sg;
            if (r < a.r_tol && sg < a.s_tol) {
                conv = true;
                break;
            }
            if (a.adapt && it < a.max_iter) {
                const double ratio = r / sg, target = a.r_tol / a.s_tol;
                double f = 1.0;
                if (ratio > 1.2 * target) f = a.tau;
                else if (ratio < 0.8 * target) f = 1.0 / a.tau;
                if (f != 1.0) {
                    for (int pr = tid; pr < mq; pr += NT) {
                        lam[pr] /= f;
                        pp[pr] /= f;
                        nu[pr] /= f;
                    }
                    T.sync();
                    if (tid < 4) rho[tid] *= f;
                    if (tid == 0) flags[1] = f;
                    T.sync();
                }
            }
        }
        for (int pr = tid; pr < mq; pr += NT) uoff[pr] = (float)(zeta[pr] + lam[pr]);
        T.sync();
    }
    const bool finished = conv || it >= a.max_iter;

    // objective (1/q) sum f(x) of eq. (2) once the instance is finished
    double obj = 0.0;
    if (finished) {
        double acc = 0.0;
        const float *F2 = ea.f2, *F1 = ea.f1, *F0 = a.f0 + I.off_e;
        const int64_t tot = (int64_t)mq * n;
        for (int64_t t = tid; t < tot; t += NT) {
            const int64_t r = t / n;
            const int k = (int)(t - r * n);
            const size_t e = (size_t)r * I.ld + k;
            const double x = ea.x[e];
            acc += (double)F2[e] * x * x + (double)F1[e] * x + (double)F0[e];
        }
        obj = team_sum<NT>(T, acc, scr) / (double)q;
    }
    const double escs = team_sum<NT>(T, (double)esc, scr);
    for (int t = tid; t < scal_size(m, q); t += NT) gscal[t] = scal[t];
    if (tid == 0) {
        out[0] = it;
        out[1] = conv ? 1.0 : 0.0;
        out[2] = r_last;
        out[3] = s_last;
        for (int t = 0; t < 7; ++t) out[4 + t] = res[t];
        if (finished) out[11] = obj;
        out[12] = 0.0;
        out[13] += escs;
        out[14] = finished ? 1.0 : 0.0;
    }
    T.sync();
}


// The whole cluster (all CTAs, NW warps each) solves instance `id`.
template <int NW, int M> __device__ void solve_instance_cluster(const BatchArgs &a, int id, double *smem)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    constexpr int NT = NW * 32;
    const int tid = threadIdx.x;
    const Team<NT> T{tid};
    const BatchInst I = a.inst[id];
    const int n = I.n, m = I.m, q = I.q, mq = m * q;
    constexpr int VW = kMixedVW;

    // this CTA's shared memory: scal | crec[2][q][m][4] | cmax[2][4] | part[8] | x1n | scr | red | uoff
    double *scal = smem;
    double *lam = scal, *zeta = scal + mq, *hh = scal + 2 * mq, *pp = scal + 3 * mq, *nu = scal + 4 * mq;
    double *x1 = scal + 5 * mq, *rho = x1 + m, *flags = rho + 4;
    double *crec = smem + scal_size(m, q);
    double *cmax = crec + 2 * (size_t)q * m * 4;
    double *part = cmax + 8;
    double *x1n = part + 8;
    double *scr = x1n + kMaxM;
    float *red = (float *)(scr + kWarpsMax * 8);
    float *uoff = red + kWarpsMax * kMaxM * 4;
    double *x0s = (double *)(uoff + ((mq + 1) / 2) * 2); // this CTA's copy of x at k = 0, [mq]

    double *gscal = a.scal + I.off_scal;
    double *out = a.out + (size_t)id * kInfo;
    const bool skip = out[14] != 0.0;
    cl.sync();
    if (skip) return; // every CTA of the cluster read the same flag
    for (int t = tid; t < scal_size(m, q); t += NT) scal[t] = gscal[t];
    T.sync();
    for (int pr = tid; pr < mq; pr += NT) uoff[pr] = (float)(zeta[pr] + lam[pr]);
    const int it0 = (int)out[0];
    T.sync();

    const ElemF32 ea = {a.f2 + I.off_e, a.f1 + I.off_e, a.g2 + I.off_e, a.g1 + I.off_e, a.g0 + I.off_e,
                        a.lo + I.off_b, a.hi + I.off_b, a.y + I.off_c,  a.x + I.off_e,  a.s + I.off_c,
                        a.mu + I.off_c, a.s_lo + I.off_c, a.mu_lo + I.off_c, n, m, q, I.ld, a.sweep, a.xmin_mode};
    const double *cc = a.c + I.off_src;
    const double *sumg0 = a.sumg0 + I.off_pair;
    const int nv = (n + VW - 1) / VW;
    unsigned esc = 0;
    bool conv = false;
    double res[7] = {out[4], out[5], out[6], out[7], out[8], out[9], out[10]};
    double r_last = out[2], s_last = out[3];
    int it = it0;
    const int it_end = a.iter_budget > 0 ? min(a.max_iter, it0 + a.iter_budget) : a.max_iter;

    while (it < it_end) {
        ++it;
        const int par = it & 1;
        const bool check = (it % a.check_every == 0) || (it == a.max_iter);
        const bool cold = flags[0] != 0.0;
        const float mu_div = (float)flags[1];
        const float rho1 = (float)rho[0], rho3 = (float)rho[2], rho4 = (float)rho[3];
        const float iq = 1.0f / (float)q;
        float fcr = 0.0f, fcs = 0.0f;
        double *recs = crec + (size_t)par * q * m * 4;
        for (int j = 0; j < q; ++j) {
            float ghi[M], glo[M], fmx[M], fmn[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                ghi[i] = 0.0f;
                glo[i] = 0.0f;
                fmx[i] = -INFINITY;
                fmn[i] = INFINITY;
            }
            double *rec = recs + (size_t)j * m * 4;
            for (int v = rank * NT + tid; v < nv; v += CL * NT)
                vec32<M, VW, false>(ea, uoff, x1, nu, j, v * VW, check, cold, mu_div, rho1, rho3, rho4, iq, ghi, glo,
                                    fmx, fmn, fcr, fcs, esc, rec);
            team_flush<NT, M>(T, rec, ghi, glo, fmx, fmn, check, m, red);
        }
        if (check) {
            double v2[2] = {(double)fcr, (double)fcs};
            team_max<NT, 2>(T, v2, scr);
            if (tid == 0) {
                cmax[par * 4 + 0] = v2[0];
                cmax[par * 4 + 1] = v2[1];
            }
        }
        if (tid == 0) flags[1] = 1.0;
        cl.sync(); // every CTA's records of this iteration are complete

        const double r1 = rho[0], r2 = rho[1], r3 = rho[2];
        const double kappa = r2 / (r1 + (double)n * r2);
        double r2m = 0.0, r3m = 0.0, s1m = 0.0, s2m = 0.0;
        for (int pr = tid; pr < mq; pr += NT) {
            const int i = pr / q, j = pr - i * q;
            const size_t off = ((size_t)j * m + i) * 4;
            double S = 0.0, dmx = -INFINITY, dmn = INFINITY;
            for (int r = 0; r < CL; ++r) {
                const double *rr = cl.map_shared_rank(recs, r) + off;
                S += rr[0];
                if (check) {
                    dmx = fmax(dmx, rr[1]);
                    dmn = fmin(dmn, rr[2]);
                }
            }
            const double x0 = cl.map_shared_rank(recs, 0)[off + 3];
            const double lm = lam[pr], zt = zeta[pr], h0 = hh[pr], p0 = pp[pr];
            const double W = (S + sumg0[pr]) - (double)n * lm;
            const double lamn = kappa * ((h0 + p0) - W);
            const double Z = W + (double)n * lamn;
            const double cz = Z - p0;
            const double hn = cz < cc[i] ? cz : cc[i];
            const double pn = p0 + (hn - Z);
            if (check) {
                r2m = fmax(r2m, fabs(lamn - lm));
                r3m = fmax(r3m, fabs(hn - Z));
                const double dl = (lamn - lm) - zt;
                s1m = fmax(s1m, fmax(fabs(dmx + dl), fabs(dmn + dl)));
                s2m = fmax(s2m, fabs(hn - h0));
            }
            lam[pr] = lamn;
            zeta[pr] = lamn - lm;
            hh[pr] = hn;
            pp[pr] = pn;
            x0s[pr] = x0;
        }
        T.sync();
        if (tid < m) {
            const int i = tid;
            double sum = 0.0;
            for (int j = 0; j < q; ++j) sum += x0s[i * q + j] - nu[i * q + j];
            x1n[i] = sum / (double)q;
        }
        T.sync();
        double r4m = 0.0;
        for (int pr = tid; pr < mq; pr += NT) {
            const int i = pr / q;
            const double x0 = x0s[pr], xn = x1n[i];
            nu[pr] = nu[pr] + (xn - x0);
            if (check) r4m = fmax(r4m, fabs(x0 - xn));
        }
        T.sync();
        if (tid < m) x1[tid] = x1n[tid];
        if (tid == 0) flags[0] = 0.0;
        T.sync();
        if (check) {
            double c1 = 0.0, c2 = 0.0;
            for (int r = 0; r < CL; ++r) {
                const double *cr = cl.map_shared_rank(cmax, r) + par * 4;
                c1 = fmax(c1, cr[0]);
                c2 = fmax(c2, cr[1]);
            }
            double v[7] = {c1, r2m, r3m, r4m, s1m, s2m, c2};
            team_max<NT, 7>(T, v, scr);
            v[0] = c1;
            v[6] = c2;
#pragma unroll
            for (int t = 0; t < 7; ++t) res[t] = v[t];
            const double r = fmax(fmax(v[0], v[1]), fmax(v[2], v[3]));
            const double sg = fmax(fmax(r1 * v[4], r2 * v[5]), r3 * v[6]);
            r_last = r;
            s_last = sg;
            if (r < a.r_tol && sg < a.s_tol) {
                conv = true;
                break;
            }
            if (a.adapt && it < a.max_iter) {
                const double ratio = r / sg, target = a.r_tol / a.s_tol;
                double f = 1.0;
                if (ratio > 1.2 * target) f = a.tau;
                else if (ratio < 0.8 * target) f = 1.0 / a.tau;
                if (f != 1.0) {
                    for (int pr = tid; pr < mq; pr += NT) {
                        lam[pr] /= f;
                        pp[pr] /= f;
                        nu[pr] /= f;
                    }
                    T.sync();
                    if (tid < 4) rho[tid] *= f;
                    if (tid == 0) flags[1] = f;
                    T.sync();
                }
            }
        }
        for (int pr = tid; pr < mq; pr += NT) uoff[pr] = (float)(zeta[pr] + lam[pr]);
        T.sync();
    }
    const bool finished = conv || it >= a.max_iter;

    // objective over this CTA's share, then summed in rank order by rank 0
    double acc = 0.0;
    if (finished) {
        const float *F2 = ea.f2, *F1 = ea.f1, *F0 = a.f0 + I.off_e;
        const int64_t tot = (int64_t)mq * n;
        for (int64_t t = (int64_t)rank * NT + tid; t < tot; t += (int64_t)CL * NT) {
            const int64_t r = t / n;
            const int k = (int)(t - r * n);
            const size_t e = (size_t)r * I.ld + k;
            const double x = ea.x[e];
            acc += (double)F2[e] * x * x + (double)F1[e] * x + (double)F0[e];
        }
    }
    acc = team_sum<NT>(T, acc, scr);
    const double escs = team_sum<NT>(T, (double)esc, scr);
    if (tid == 0) {
        part[0] = acc;
        part[1] = escs;
    }
    cl.sync();
    if (rank == 0) {
        for (int t = tid; t < scal_size(m, q); t += NT) gscal[t] = scal[t];
        if (tid == 0) {
            double obj = 0.0, es = 0.0;
            for (int r = 0; r < CL; ++r) {
                obj += cl.map_shared_rank(part, r)[0];
                es += cl.map_shared_rank(part, r)[1];
            }
            out[0] = it;
            out[1] = conv ? 1.0 : 0.0;
            out[2] = r_last;
            out[3] = s_last;
            for (int t = 0; t < 7; ++t) out[4 + t] = res[t];
            if (finished) out[11] = obj / (double)q;
            out[12] = 0.0;
            out[13] += es;
            out[14] = finished ? 1.0 : 0.0;
        }
    }
    cl.sync(); // rank 0 has read every CTA's shared memory
}

template <int NW, int M> __global__ void __launch_bounds__(NW * 32, 16 / NW) batch_kernel(BatchArgs a)
{
    extern __shared__ double smem[];
    __shared__ int s_item;
    const int nX = a.nLS ? a.nLS[0] : a.nX, nL = a.nLS ? a.nLS[1] : a.nL, nS = a.nLS ? a.nLS[2] : a.nS;
    // Largest instances: the whole cluster is one team (rank 0 takes the item
    // and the other CTAs read it through distributed shared memory).
    if (nX > 0) {
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        for (;;) {
            if (cl.block_rank() == 0 && threadIdx.x == 0) s_item = atomicAdd(a.qX, 1);
            cl.sync();
            const int item = *cl.map_shared_rank(&s_item, 0);
            cl.sync();
            if (item >= nX) break;
            solve_instance_cluster<NW, M>(a, a.orderX[item], smem);
        }
    }
    // Large instances: the whole CTA is one team.
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.qL, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nL) break;
        solve_instance<NW * 32, M>(a, a.orderL[item], smem, threadIdx.x);
    }
    // Small instances: each warp is a team with its own slice.
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *slice = smem + (size_t)w * a.slice_doubles;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.qS, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= nS) break;
        solve_instance<32, M>(a, a.orderS[item], slice, lane);
    }
}

template <int NW> void *batch_fn(int mb)
{
    switch (mb) {
    case 2: return (void *)batch_kernel<NW, 2>;
    case 4: return (void *)batch_kernel<NW, 4>;
    default: return (void *)batch_kernel<NW, 8>;
    }
}

void *batch_pick(int warps, int mb)
{
    switch (warps) {
    case 4: return batch_fn<4>(mb);
    case 16: return batch_fn<16>(mb);
    default: return batch_fn<8>(mb);
    }
}

// Receding-horizon warm start (Sec. II, Alg. 2): the previous solution of a
// controller moved one step forward in place (x_k <- x_{k+1}, last step
// kept; the same for s and mu), x_1^(i) reset to the mean of the new first
// moves, cold flag cleared.  One CTA per instance.
__global__ void shift_state_kernel(const BatchInst *inst, const int *ids, int count, float *x, float *s, float *s_lo,
                                   float *mu, float *mu_lo, double *scal)
{
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        const BatchInst I = inst[ids[t]];
        const int n = I.n, rows_e = I.m * I.q;
        // rows of x, then rows of s, s_lo, mu, mu_lo; each shifted left by one
        for (int r = 0; r < rows_e + 4 * I.q; ++r) {
            float *row;
            if (r < rows_e) row = x + I.off_e + (int64_t)r * I.ld;
            else {
                const int c = (r - rows_e) / I.q, j = (r - rows_e) % I.q;
                float *base = c == 0 ? s : (c == 1 ? s_lo : (c == 2 ? mu : mu_lo));
                row = base + I.off_c + (int64_t)j * I.ld;
            }
            for (int k0 = 0; k0 < n - 1; k0 += blockDim.x) {
                const int k = k0 + threadIdx.x;
                const float v = k < n - 1 ? row[k + 1] : 0.0f;
                __syncthreads();
                if (k < n - 1) row[k] = v;
                __syncthreads();
            }
        }
        double *sc = scal + I.off_scal;
        const int mq = I.m * I.q;
        if (threadIdx.x < I.m) {
            const int i = threadIdx.x;
            double sum = 0.0;
            for (int j = 0; j < I.q; ++j) sum += (double)x[I.off_e + ((int64_t)i * I.q + j) * I.ld];
            sc[5 * mq + i] = sum / (double)I.q;
        }
        if (threadIdx.x == 0) sc[5 * mq + I.m + 4] = 0.0;
        __syncthreads();
    }
}

// Receding-horizon step request: the whole instance (coefficients, bounds,
// demand, x, s, mu) moves one step forward in place; the new last step's
// data comes from `payload` (per instance, FP32: f2 f1 f0 g2 g1 g0 [m][q],
// lo hi [m], y [q]); x at the new last step is clamped to its new bounds;
// sum_k beta_0 is recomputed; x_1^(i) = mean of the new first moves; cold
// flag cleared.  One CTA per instance.
__global__ void shift_step_kernel(const BatchInst *inst, const int *ids, int count, const float *payload,
                                  int payload_stride, float *f2, float *f1, float *f0, float *g2, float *g1, float *g0,
                                  float *lo, float *hi, float *y, float *x, float *s, float *s_lo, float *mu,
                                  float *mu_lo, double *sumg0, double *scal)
{
    for (int t = blockIdx.x; t < count; t += gridDim.x) {
        const int id = ids[t];
        const BatchInst I = inst[id];
        const int n = I.n, m = I.m, q = I.q, mq = m * q;
        const float *pl = payload + (size_t)id * payload_stride;
        float *erows[7] = {f2, f1, f0, g2, g1, g0, x};
        float *crows[5] = {y, s, s_lo, mu, mu_lo};
        const int nrows = 7 * mq + 2 * m + 5 * q;
        for (int r = 0; r < nrows; ++r) {
            float *row;
            if (r < 7 * mq) row = erows[r / mq] + I.off_e + (int64_t)(r % mq) * I.ld;
            else if (r < 7 * mq + 2 * m) {
                const int rr = r - 7 * mq;
                row = (rr < m ? lo : hi) + I.off_b + (int64_t)(rr % m) * I.ld;
            } else {
                const int rr = r - 7 * mq - 2 * m;
                row = crows[rr / q] + I.off_c + (int64_t)(rr % q) * I.ld;
            }
            for (int k0 = 0; k0 < n - 1; k0 += blockDim.x) {
                const int k = k0 + threadIdx.x;
                const float v = k < n - 1 ? row[k + 1] : 0.0f;
                __syncthreads();
                if (k < n - 1) row[k] = v;
                __syncthreads();
            }
        }
        // the new last step
        const int last = n - 1;
        for (int u = threadIdx.x; u < mq; u += blockDim.x) {
            const int64_t e = I.off_e + (int64_t)u * I.ld + last;
            f2[e] = pl[0 * mq + u];
            f1[e] = pl[1 * mq + u];
            f0[e] = pl[2 * mq + u];
            g2[e] = pl[3 * mq + u];
            g1[e] = pl[4 * mq + u];
            g0[e] = pl[5 * mq + u];
        }
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            lo[I.off_b + (int64_t)i * I.ld + last] = pl[6 * mq + i];
            hi[I.off_b + (int64_t)i * I.ld + last] = pl[6 * mq + m + i];
        }
        for (int j = threadIdx.x; j < q; j += blockDim.x) y[I.off_c + (int64_t)j * I.ld + last] = pl[6 * mq + 2 * m + j];
        __syncthreads();
        for (int u = threadIdx.x; u < mq; u += blockDim.x) {
            const int i = u / q;
            const int64_t e = I.off_e + (int64_t)u * I.ld + last;
            const float l = lo[I.off_b + (int64_t)i * I.ld + last], h = hi[I.off_b + (int64_t)i * I.ld + last];
            x[e] = x[e] < l ? l : (x[e] > h ? h : x[e]);
        }
        // sum_k beta_0 per pair (one warp per pair, fixed order)
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int u = w; u < mq; u += nw) {
            double acc = 0.0;
            for (int k = lane; k < n; k += 32) acc += (double)g0[I.off_e + (int64_t)u * I.ld + k];
            acc = warp_sum(acc);
            if (lane == 0) sumg0[I.off_pair + u] = acc;
        }
        __syncthreads();
        double *sc = scal + I.off_scal;
        if (threadIdx.x < m) {
            const int i = threadIdx.x;
            double sum = 0.0;
            for (int j = 0; j < q; ++j) sum += (double)x[I.off_e + ((int64_t)i * q + j) * I.ld];
            sc[5 * mq + i] = sum / (double)q;
        }
        if (threadIdx.x == 0) sc[5 * mq + m + 4] = 0.0;
        __syncthreads();
    }
}

} // namespace

void launch_shift_step(const BatchInst *inst, const int *ids, int count, const float *payload, int payload_stride,
                       float *f2, float *f1, float *f0, float *g2, float *g1, float *g0, float *lo, float *hi,
                       float *y, float *x, float *s, float *s_lo, float *mu, float *mu_lo, double *sumg0,
                       double *scal, cudaStream_t st)
{
    if (count > 0)
        shift_step_kernel<<<std::min(count, 1024), 256, 0, st>>>(inst, ids, count, payload, payload_stride, f2, f1, f0,
                                                                 g2, g1, g0, lo, hi, y, x, s, s_lo, mu, mu_lo, sumg0,
                                                                 scal);
}

void launch_shift_state(const BatchInst *inst, const int *ids, int count, float *x, float *s, float *s_lo, float *mu,
                        float *mu_lo, double *scal, cudaStream_t st)
{
    if (count > 0) shift_state_kernel<<<std::min(count, 1024), 256, 0, st>>>(inst, ids, count, x, s, s_lo, mu, mu_lo, scal);
}

size_t batch_slice_doubles(int max_m, int max_q)
{
    const int mq = max_m * max_q;
    size_t d = (size_t)scal_size(max_m, max_q) + (size_t)max_q * max_m * 4 + kMaxM + kWarpsMax * 8 +
               (kWarpsMax * kMaxM * 4 + 1) / 2 + (mq + 1) / 2 + 8;
    return (d + 3) / 4 * 4;
}

size_t batch_cluster_team_doubles(int max_m, int max_q)
{
    const int mq = max_m * max_q;
    return (size_t)scal_size(max_m, max_q) + 2 * (size_t)max_q * max_m * 4 + 16 + kMaxM + kWarpsMax * 8 +
           (kWarpsMax * kMaxM * 4 + 1) / 2 + (mq + 1) / 2 + mq + 8;
}

size_t batch_smem_bytes(int warps, size_t slice_doubles)
{
    return sizeof(double) * slice_doubles * (size_t)warps;
}

int batch_blocks_per_sm(int warps, int mb, size_t smem)
{
    void *fn = batch_pick(warps, mb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, warps * 32, smem) != cudaSuccess) return 0;
    return nb;
}

// The kernel's shared-memory attribute is set by batch_blocks_per_sm, which
// the host calls before launching (and before any graph capture).
cudaError_t launch_batch(int warps, int mb, int grid, int cluster, const BatchArgs &a, size_t smem, cudaStream_t st)
{
    void *fn = batch_pick(warps, mb);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster > 1 ? cluster : 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&a};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

int batch_max_clusters(int warps, int mb, int cluster, size_t smem)
{
    void *fn = batch_pick(warps, mb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cluster > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * 152);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) return 0;
    return nc;
}

} // namespace admm_impl

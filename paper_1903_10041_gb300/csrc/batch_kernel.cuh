// Batched solve: thousands of independent instances of uneven n, m, q in one
// persistent launch (mixed precision).
//
// Each instance is solved by one team of threads that runs the ADMM loop of
// App. A for it with team-local synchronisation only: a thread-block
// cluster, a whole CTA, or a single warp (so a CTA of W warps holds W small
// instances at once), by size thresholds.  Teams take work from three
// global queues of instance ids (cluster, CTA, warp teams), each sorted by
// decreasing estimated work (longest-processing-time order), so a team that
// finishes early takes the next instance.  Each instance stops on its own
// stop test.
//
// A cluster team (2-8 CTAs on neighbouring SMs): each CTA reduces its part
// of every row into records in its own shared memory, one hardware cluster
// barrier per iteration follows, and every CTA reads all CTAs' records
// through distributed shared memory in rank order and runs the scalar steps
// redundantly.
//
// Per iteration a team splits the q rows of nv column pairs of its instance
// into W equal contiguous ranges, one per warp (W warps in the team); a
// warp walks its range row piece by row piece, its lanes taking
// consecutive column pairs (coalesced) and running the element update of
// mixed_elem.cuh; each piece is reduced by shuffles into a record in shared
// memory, one team barrier follows, and the per-(i, j) scalar steps,
// residuals and stop test run on the team.  The arithmetic and its order
// depend only on the instance's own shape and its team kind (fixed by the
// instance's size), so an instance gives the same bits alone and in any mix.
//
// An iteration budget lets a launch stop every instance after a given
// number of iterations with its state saved; the serving loop uses it (with
// time-balanced budgets and round-robin slices, batch.h) to run the batch in
// ticks and admit new instances between ticks.
#pragma once
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

// Team-wide FP64 sum over NT threads of one CTA (fixed order), every thread gets the result.
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

enum { TEAM_WARP = 0, TEAM_CTA = 1, TEAM_CLUSTER = 2 };

// Column pairs per warp of a team of W warps over P = q nv pairs: equal
// shares in whole lane rounds.  Warp w takes pairs [w chunk, (w + 1) chunk)
// of the row-major pair index j nv + v, so rows j touch warps
// j nv / chunk .. ((j + 1) nv - 1) / chunk, and the record of (row j, warp
// w) sits at index j + w: rows share at most their boundary warp, so the
// indices never collide and stay below q + W - 1.
__host__ __device__ inline int64_t team_chunk(int W, int q, int nv)
{
    const int64_t P = (int64_t)q * nv;
    return ((P + W - 1) / W + 31) / 32 * 32;
}

// One team solves instance `id` from its saved state until it stops or the
// iteration budget runs out.  KIND: one warp (slice = that warp's shared
// memory), one CTA, or a thread-block cluster (every CTA runs this
// function; each holds a copy of the scalar state and records of the row
// pieces its warps processed).  Work per iteration: each warp its range of
// column pairs, piece by piece, reducing each piece with shuffles only; one
// team barrier; then the per-(i, j) scalar steps read the records of each
// row in warp order.
template <int KIND, int NW, int M, bool ROLL> __device__ void solve_team(const BatchArgs &a, int id, double *smem)
{
    namespace cg = cooperative_groups;
    constexpr int NTL = KIND == TEAM_WARP ? 32 : NW * 32; // threads of this CTA in the team
    constexpr int NWT = NTL / 32;
    constexpr int VW = kMixedVW;
    const int lane = threadIdx.x & 31;
    const int tid = KIND == TEAM_WARP ? lane : (int)threadIdx.x;
    const int wl = KIND == TEAM_WARP ? 0 : (int)(threadIdx.x >> 5);
    int CL = 1, rank = 0;
    if constexpr (KIND == TEAM_CLUSTER) {
        CL = (int)cg::this_cluster().num_blocks();
        rank = (int)cg::this_cluster().block_rank();
    }
    const Team<NTL> T{tid};
    auto sync_local = [&]() {
        if constexpr (KIND == TEAM_WARP) __syncwarp();
        else __syncthreads();
    };
    auto sync_team = [&]() {
        if constexpr (KIND == TEAM_CLUSTER) cg::this_cluster().sync();
        else sync_local();
    };

    const BatchInst I = a.inst[id];
    const int n = I.n, m = I.m, q = I.q, mq = m * q;
    const int nv = (n + VW - 1) / VW;
    const int W = NWT * CL, gw = rank * NWT + wl;
    // inputs staged in shared memory by cp.async (CTA and cluster teams of the m <= 4 kernel): the
    // rolling stage of every input (ROLL: batches, where an instance stays with its team), else the
    // double stage of the read-only coefficients (serving, whose round-robin slices can bring an
    // instance back to an SM with stale L1 lines).  Both give the same bits.
    constexpr bool STG = KIND != TEAM_WARP && M == 4;
    float2 *stage = (float2 *)((char *)smem + a.stage_off);
    const int64_t chunk = team_chunk(W, q, nv);
    const int64_t npairs = (int64_t)q * nv;
    const int items = q + W - 1; // record slots: (row j, warp w) at j + w

    // shared memory: scal | rec[2][items][m][4] | cmax[2][NWT][2] | part[24] | x0s[mq] | x1n | scr | uoff | x1nu
    // part: [0], [1] end-of-solve sums; [2] kappa; [3] the adaptation factor of a check; [16..19] fpar;
    // [20..23] ipar.  Thread 0 keeps these team-wide values current so that the other threads read them
    // instead of each converting and dividing on the FP64 pipe.
    double *scal = smem;
    double *lam = scal, *zeta = scal + mq, *hh = scal + 2 * mq, *pp = scal + 3 * mq, *nu = scal + 4 * mq;
    double *x1 = scal + 5 * mq, *rho = x1 + m, *flags = rho + 4;
    double *rec0 = smem + scal_size(m, q);
    double *cmax = rec0 + 2 * (size_t)items * m * 4;
    double *part = cmax + 4 * NWT;
    float *fpar = (float *)(part + 16); // rho_1, rho_3, rho_4 and the pending mu divisor, in FP32
    int *ipar = (int *)(part + 20);     // converged, penalties changed, cold start
    double *x0s = part + 24;
    double *x1n = x0s + mq;
    double *scr = x1n + kMaxM;
    float *uoff = (float *)(scr + kWarpsMax * 8); // [mq] (float)(zeta + lambda)
    float *x1nu = uoff + mq;                      // [mq] (float)(x1 + nu)

    double *gscal = a.scal + I.off_scal;
    double *out = a.out + (size_t)id * kInfo;
    const bool skip = __ldcg(out + 14) != 0.0;
    sync_team();
    if (skip) return; // every member read the same flag
    for (int t = tid; t < scal_size(m, q); t += NTL) scal[t] = __ldcg(gscal + t);
    sync_local();
    for (int pr = tid; pr < mq; pr += NTL) {
        uoff[pr] = (float)(zeta[pr] + lam[pr]);
        x1nu[pr] = (float)(x1[pr / q] + nu[pr]);
    }
    if (tid == 0) {
        part[2] = rho[1] / (rho[0] + (double)n * rho[1]); // kappa of step (b)
        fpar[0] = (float)rho[0];
        fpar[1] = (float)rho[2];
        fpar[2] = (float)rho[3];
        fpar[3] = (float)flags[1];
        ipar[2] = flags[0] != 0.0;
    }
    const int it0 = (int)__ldcg(out);
    sync_local();

    // the arrays' bases and this instance's 32-bit offsets into them (the arrays hold < 2^32 elements)
    const ElemF32T<unsigned> ea = {a.f2, a.f1, a.g2, a.g1, a.g0, a.lo, a.hi, a.y, a.x, a.s, a.mu, a.s_lo, a.mu_lo,
                                   n, m, q, I.ld, a.sweep, a.xmin_mode, q, 1, a.dbg,
                                   (unsigned)I.off_e, (unsigned)I.off_b, (unsigned)I.off_c};
    const double *cc = a.c + I.off_src;
    const double *sumg0 = a.sumg0 + I.off_pair;
    unsigned esc = 0;
    bool conv = false;
    double res[7];
    for (int t = 0; t < 7; ++t) res[t] = __ldcg(out + 4 + t);
    double r_last = __ldcg(out + 2), s_last = __ldcg(out + 3);
    int it = it0;
    int budget = a.iter_budget;
    if (budget > 0 && a.tick_work) {
        float cost = team_iter_cost(n, m, q, W * 32);
        // a cluster team takes its instance once per tick: its one pass stands for the R
        // round-robin slices a CTA team's instance gets
        if constexpr (KIND == TEAM_CLUSTER)
            if (a.tick_rounds) cost /= (float)max(1, *a.tick_rounds);
        budget = (int)fminf(fmaxf(*a.tick_work / cost, 1.0f), 1.0e9f);
    }
    const int it_end = budget > 0 ? (int)min((int64_t)a.max_iter, (int64_t)it0 + budget) : a.max_iter;

    while (it < it_end) {
        ++it;
        const int par = it & 1;
        const bool check = (it % a.check_every == 0) || (it == a.max_iter);
        const bool cold = ipar[2] != 0;
        const float mu_div = fpar[3];
        const float rho1 = fpar[0], rho3 = fpar[1], rho4 = fpar[2];
        const float iq = 1.0f / (float)q;
        // lane maxima and minima that only check iterations use: with the staged
        // (m <= 4) update they live in the thread's own shared-memory slots (11
        // floats apart, no bank conflicts) instead of registers across the loop
        float fcr_r = 0.0f, fcs_r = 0.0f;
        float *px = (float *)(stage + NWT * stage_region_slots<M>() * 32) + tid * 11;
        float &fcr = *(STG ? px + 2 * M : &fcr_r);
        float &fcs = *(STG ? px + 2 * M + 1 : &fcs_r);
        fcr = 0.0f;
        fcs = 0.0f;
        double *recs = rec0 + (size_t)par * items * m * 4;
        const int64_t pend = min(npairs, (int64_t)(gw + 1) * chunk);
        for (int64_t pa = (int64_t)gw * chunk; pa < pend;) {
            const int j = (int)(pa / nv);
            const int v0 = (int)(pa - (int64_t)j * nv);
            const int v1 = (int)(min(pend, (int64_t)(j + 1) * nv) - (int64_t)j * nv);
            pa = (int64_t)j * nv + v1;
            float2 ghi[M], glo[M]; // per-lane capacity sums of the column pairs
            float fmx_r[M], fmn_r[M];
            float *fmx = STG ? px : fmx_r, *fmn = STG ? px + M : fmn_r;
#pragma unroll
            for (int i = 0; i < M; ++i) {
                ghi[i] = make_float2(0.0f, 0.0f);
                glo[i] = make_float2(0.0f, 0.0f);
                if (!STG || check) {
                    fmx[i] = -INFINITY;
                    fmn[i] = INFINITY;
                }
            }
            double *rec = recs + (size_t)(j + gw) * m * 4;
            if constexpr (STG && ROLL) {
                // one rolling stage per warp, each slot group refilled for round r + 1 as round r reads it
                float2 *stw = stage + (size_t)wl * stage_region_slots<M>() * 32 + lane;
                int v = v0 + lane;
                roll_prologue<M>(ea, j, v * VW, v < v1, stw);
                for (; v < v1; v += 32) {
                    const int kn = v + 32 < v1 ? (v + 32) * VW : -1;
                    vec32<M, VW, false, STAGE_ROLL>(ea, uoff, x1nu, j, v * VW, check, cold, mu_div, rho1, rho3,
                                                    rho4, iq, ghi, glo, fmx, fmn, fcr, fcs, esc, rec, stw, kn);
                }
                cp_async_wait0();
            } else if constexpr (STG) {
                // two stages per warp; round r of the piece reads stage r & 1
                // while the copies of round r + 1 fill the other
                float2 *stw = stage + (size_t)wl * stage_region_slots<M>() * 32 + lane;
                int v = v0 + lane;
                if (v < v1) stage_vec32<M>(ea, j, v * VW, stw);
                cp_async_commit();
                for (int r = 0; v < v1; v += 32, ++r) {
                    float2 *cur = stw + (r & 1) * stage_slots<M>() * 32;
                    if (v + 32 < v1) {
                        stage_vec32<M>(ea, j, (v + 32) * VW, stw + ((r + 1) & 1) * stage_slots<M>() * 32);
                        prefetch_mutable<M>(ea, j, (v + 32) * VW);
                    }
                    cp_async_commit();
                    cp_async_wait1(); // this round's copies have landed
                    vec32<M, VW, false, STAGE_DOUBLE>(ea, uoff, x1nu, j, v * VW, check, cold, mu_div, rho1, rho3, rho4,
                                              iq, ghi, glo, fmx, fmn, fcr, fcs, esc, rec, cur);
                }
                cp_async_wait0();
            } else {
                for (int v = v0 + lane; v < v1; v += 32) {
                    if (v + 32 < v1) prefetch_vec32<M>(ea, j, (v + 32) * VW, cold);
                    vec32<M, VW, false>(ea, uoff, x1nu, j, v * VW, check, cold, mu_div, rho1, rho3, rho4, iq, ghi,
                                        glo, fmx, fmn, fcr, fcs, esc, rec);
                }
            }
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (i < m) {
                    FF v = lanes_sum(ghi[i], glo[i]);
                    float hi = check ? fmx[i] : 0.0f, lo = check ? fmn[i] : 0.0f;
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
                        rec[i * 4 + 0] = (double)v.hi + (double)v.lo;
                        rec[i * 4 + 1] = check ? (double)hi : 0.0;
                        rec[i * 4 + 2] = check ? (double)lo : 0.0;
                    }
                }
        }
        if (check) {
            const float wr = warp_max(fcr), ws = warp_max(fcs);
            if (lane == 0) {
                cmax[(par * NWT + wl) * 2 + 0] = (double)wr;
                cmax[(par * NWT + wl) * 2 + 1] = (double)ws;
            }
        }
        sync_team(); // every record of this iteration is complete and visible
        if (tid == 0) { // the pending mu rescale has been applied (every thread read it before the barrier)
            flags[1] = 1.0;
            fpar[3] = 1.0f;
        }

        const double kappa = part[2];
        double r2m = 0.0, r3m = 0.0, s1m = 0.0, s2m = 0.0;
        for (int pr = tid; pr < mq; pr += NTL) {
            const int i = pr / q, j = pr - i * q;
            double Ssum = 0.0, dmx = -INFINITY, dmn = INFINITY, x0 = 0.0;
            const int wf = (int)((int64_t)j * nv / chunk), wlst = (int)(((int64_t)j * nv + nv - 1) / chunk);
            for (int w = wf; w <= wlst; ++w) { // the warps whose ranges cover row j, in order
                const double *rb = recs;
                if constexpr (KIND == TEAM_CLUSTER) rb = cg::this_cluster().map_shared_rank(recs, w / NWT);
                const double *rr = rb + ((size_t)(j + w) * m + i) * 4;
                Ssum += rr[0];
                if (check) {
                    dmx = fmax(dmx, rr[1]);
                    dmn = fmin(dmn, rr[2]);
                }
                if (w == wf) x0 = (double)*(const float *)(rr + 3); // k = 0 lies in the first warp's piece
            }
            const double lm = lam[pr], zt = zeta[pr], h0 = hh[pr], p0 = pp[pr];
            const double Wv = (Ssum + sumg0[pr]) - (double)n * lm;
            const double lamn = kappa * ((h0 + p0) - Wv);
            const double Z = Wv + (double)n * lamn;
            const double cz = Z - p0;
            const double hn = cz < cc[i] ? cz : cc[i];
            const double pn = p0 + (hn - Z);
            if (check) {
                r2m = max_nonneg(r2m, fabs(lamn - lm));
                r3m = max_nonneg(r3m, fabs(hn - Z));
                const double dl = (lamn - lm) - zt;
                s1m = max_nonneg(s1m, max_nonneg(fabs(dmx + dl), fabs(dmn + dl)));
                s2m = max_nonneg(s2m, fabs(hn - h0));
            }
            lam[pr] = lamn;
            zeta[pr] = lamn - lm;
            hh[pr] = hn;
            pp[pr] = pn;
            x0s[pr] = x0;
        }
        sync_local();
        for (int i = tid >> 5; i < m; i += NTL / 32) { // (c), mean over j: one warp per source
            const int lane = tid & 31;
            double sum = 0.0;
            for (int j = lane; j < q; j += 32) sum += x0s[i * q + j] - nu[i * q + j];
            sum = warp_sum(sum);
            if (lane == 0) x1n[i] = sum / (double)q;
        }
        sync_local();
        // (h), and the FP32 offsets of the next element phase (lambda, zeta final; x1 = x1n)
        double r4m = 0.0;
        for (int pr = tid; pr < mq; pr += NTL) {
            const int i = pr / q;
            const double x0 = x0s[pr], xn = x1n[i];
            const double nun = nu[pr] + (xn - x0);
            nu[pr] = nun;
            uoff[pr] = (float)(zeta[pr] + lam[pr]);
            x1nu[pr] = (float)(xn + nun);
            if (check) r4m = max_nonneg(r4m, fabs(x0 - xn));
        }
        if (tid < m) x1[tid] = x1n[tid];
        if (tid == 0) {
            flags[0] = 0.0;
            ipar[2] = 0;
        }
        sync_local();
        if (check) {
            // maxima of the residual terms: per warp, then over the team's warps and (for a cluster)
            // the CTAs' column maxima by thread 0, which takes the stop decision and the adaptation
            // of Sec. IV-A and passes them on; every CTA of a cluster decides the same way
            double v[5] = {r2m, r3m, r4m, s1m, s2m};
#pragma unroll
            for (int t = 0; t < 5; ++t) v[t] = warp_max_nonneg(v[t]);
            if constexpr (KIND != TEAM_WARP) {
                if (lane == 0)
                    for (int t = 0; t < 5; ++t) scr[wl * 8 + t] = v[t];
                sync_local();
            }
            if (tid == 0) {
                double w[7] = {0.0, v[0], v[1], v[2], v[3], v[4], 0.0};
                if constexpr (KIND != TEAM_WARP)
                    for (int ww = 0; ww < NWT; ++ww)
                        for (int t = 0; t < 5; ++t) w[1 + t] = max_nonneg(w[1 + t], scr[ww * 8 + t]);
                for (int r = 0; r < CL; ++r) {
                    const double *cb = cmax;
                    if constexpr (KIND == TEAM_CLUSTER) cb = cg::this_cluster().map_shared_rank(cmax, r);
                    for (int ww = 0; ww < NWT; ++ww) {
                        w[0] = max_nonneg(w[0], cb[(par * NWT + ww) * 2 + 0]);
                        w[6] = max_nonneg(w[6], cb[(par * NWT + ww) * 2 + 1]);
                    }
                }
                for (int t = 0; t < 7; ++t) res[t] = w[t];
                const double r = fmax(fmax(w[0], w[1]), fmax(w[2], w[3]));
                const double sgm = fmax(fmax(rho[0] * w[4], rho[1] * w[5]), rho[2] * w[6]);
                r_last = r;
                s_last = sgm;
                const bool cv = r < a.r_tol && sgm < a.s_tol;
                double f = 1.0;
                if (!cv && a.adapt && it < a.max_iter && it >= a.adapt_start) { // Sec. IV-A, duals rescaled
                    const double ratio = r / sgm, target = a.adapt_target;
                    if (ratio > 1.2 * target) f = a.tau;
                    else if (ratio < 0.8 * target) f = 1.0 / a.tau;
                }
                ipar[0] = cv;
                ipar[1] = f != 1.0;
                part[3] = f;
            }
            sync_local();
            if (ipar[0]) {
                conv = true;
                break;
            }
            if (ipar[1]) {
                const double f = part[3];
                for (int pr = tid; pr < mq; pr += NTL) {
                    lam[pr] /= f;
                    pp[pr] /= f;
                    nu[pr] /= f;
                    uoff[pr] = (float)(zeta[pr] + lam[pr]);
                    x1nu[pr] = (float)(x1[pr / q] + nu[pr]);
                }
                if (tid == 0) {
                    for (int t = 0; t < 4; ++t) rho[t] *= f;
                    flags[1] = f;
                    part[2] = rho[1] / (rho[0] + (double)n * rho[1]);
                    fpar[0] = (float)rho[0];
                    fpar[1] = (float)rho[2];
                    fpar[2] = (float)rho[3];
                    fpar[3] = (float)f;
                }
                sync_local();
            }
        }
    }
    const bool finished = conv || it >= a.max_iter;

    // objective (1/q) sum f(x) of eq. (2): each CTA sums its share, rank 0 adds in rank order
    double acc = 0.0;
    if (finished) {
        const float *F2 = a.f2 + I.off_e, *F1 = a.f1 + I.off_e, *F0 = a.f0 + I.off_e, *X = a.x + I.off_e;
        const int64_t tot = (int64_t)mq * n;
        for (int64_t t = (int64_t)rank * NTL + tid; t < tot; t += (int64_t)CL * NTL) {
            const int64_t r = t / n;
            const int k = (int)(t - r * n);
            const size_t e = ADMM_IDX((size_t)r * I.ld + k, 1, ea.len_x(), a.dbg, DBG_X);
            const double x = X[e];
            acc += (double)F2[e] * x * x + (double)F1[e] * x + (double)F0[e];
        }
    }
    acc = team_sum<NTL>(T, acc, scr);
    const double escs = team_sum<NTL>(T, (double)esc, scr);
    if (tid == 0) {
        part[0] = acc;
        part[1] = escs;
    }
    sync_team();
    if (rank == 0) {
        for (int t = tid; t < scal_size(m, q); t += NTL) gscal[t] = scal[t];
        if (tid == 0) {
            double obj = 0.0, es = 0.0;
            for (int r = 0; r < CL; ++r) {
                const double *pb = part;
                if constexpr (KIND == TEAM_CLUSTER) pb = cg::this_cluster().map_shared_rank(part, r);
                obj += pb[0];
                es += pb[1];
            }
            out[0] = it;
            out[1] = conv ? 1.0 : 0.0;
            out[2] = r_last;
            out[3] = s_last;
            for (int t = 0; t < 7; ++t) out[4 + t] = res[t];
            if (finished) out[11] = obj / (double)q;
            out[12] = 0.0;
            out[13] = __ldcg(out + 13) + es;
            out[14] = finished ? 1.0 : 0.0;
        }
    }
    sync_team(); // rank 0 has read every member's shared memory
}

template <int NW, int M, bool ROLL> __global__ void __launch_bounds__(NW * 32, 16 / NW) batch_kernel(BatchArgs a)
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
            solve_team<TEAM_CLUSTER, NW, M, ROLL>(a, a.orderX[item], smem);
        }
    }
    const int R = a.tick_rounds ? max(1, *a.tick_rounds) : 1;
    // Large instances: the whole CTA is one team.  id -1: the instance is
    // being run by another team (round-robin launches only).
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = atomicAdd(a.qL, 1);
            int id = item < nL * R ? a.orderL[item % max(nL, 1)] : -2;
            if (id >= 0 && R > 1) {
                if (atomicCAS(a.lock + id, 0, 1) != 0) id = -1;
                else __threadfence();
            }
            s_item = id;
        }
        __syncthreads();
        const int id = s_item;
        __syncthreads();
        if (id == -2) break;
        if (id < 0) continue;
        solve_team<TEAM_CTA, NW, M, ROLL>(a, id, smem);
        if (R > 1) {
            __syncthreads(); // every thread's state writes precede the release
            if (threadIdx.x == 0) {
                __threadfence();
                atomicExch(a.lock + id, 0);
            }
        }
    }
    // Small instances: each warp is a team with its own slice.
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *slice = smem + (size_t)w * a.slice_doubles;
    for (;;) {
        int id = 0;
        if (lane == 0) {
            const int item = atomicAdd(a.qS, 1);
            id = item < nS * R ? a.orderS[item % max(nS, 1)] : -2;
            if (id >= 0 && R > 1) {
                if (atomicCAS(a.lock + id, 0, 1) != 0) id = -1;
                else __threadfence();
            }
        }
        id = __shfl_sync(0xffffffffu, id, 0);
        if (id == -2) break;
        if (id < 0) continue;
        solve_team<TEAM_WARP, NW, M, ROLL>(a, id, slice);
        if (R > 1) {
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicExch(a.lock + id, 0);
            }
        }
    }
}

} // namespace

} // namespace admm_impl

// admm_solve_noalloc: the single-instance solve for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc or any allocating routine: code that
// runs inside a host callback or a real-time control loop where an allocation
// may block or fail, embedded controllers with a fixed memory budget set at
// start-up, and plugins whose host application owns every device
// allocation.  For them this entry point takes every input and output from
// the caller and keeps the solver's scratch (partial sums, barrier counter,
// status word, scalar state, per-solve record) in one file-scope device
// array of fixed size.  It runs the same persistent solve kernel as
// admm_solve, with the same arithmetic.
//
// The array is part of the library image, so every GPU that loads the
// library holds it until the process exits.  Its device address is looked
// up once per device (cudaGetSymbolAddress with that device current) on the
// first call made on that device; make that first call before any stream
// capture.  All calls share the array and it keeps the last call's
// contents: each call clears what must start at zero, and calls that
// overlap on the GPU (from several host threads or streams at once) race
// on it and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

using namespace admm_impl;

namespace {

constexpr size_t kScratchDoubles = 512 * 1024; // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Error paths only: the message goes to admm_last_error().
admm_status nfail(admm_status s, const char *msg, const char *detail = "")
{
    char buf[512];
    snprintf(buf, sizeof buf, "admm_solve_noalloc: %s%s", msg, detail);
    set_last_error(buf);
    return s;
}

// Validation of the caller's problem and preparation of the scratch: the
// scalar state vector, sum_k beta_0 per pair, zeroed counters.  One CTA per
// pair; all CTAs also scan the elements for invalid data.  It reads the
// caller's arrays and writes only the scratch, so a problem found invalid
// leaves the caller's state as it was.
__global__ void noalloc_prepare(int n, int m, int q, const double *f2, const double *f1, const double *f0,
                                const double *g2, const double *g1, const double *g0, const double *lo,
                                const double *hi, const double *y, const double *c, const double *lam,
                                const double *zeta, const double *hh,
                                const double *pp, const double *nu, const double *x1, double rho1, double rho2,
                                double rho3, double rho4, int cold, double *scal, double *sumg0,
                                unsigned *bar, int *status, unsigned *flags)
{
    const int mq = m * q;
    const int pr = blockIdx.x, i = pr / q, j = pr - i * q;
    __shared__ double sh[2][32];
    // element scan of this pair's row (and its bound / demand rows)
    unsigned bits = 0;
    double s0 = 0.0, smin = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const size_t e = (size_t)pr * n + k;
        const double v[6] = {f2[e], f1[e], f0[e], g2[e], g1[e], g0[e]};
        for (int u = 0; u < 6; ++u)
            if (!isfinite(v[u])) bits |= 1u;
        if (v[0] < 0.0 || v[3] < 0.0) bits |= 2u;
        const double l = lo[(size_t)i * n + k], h = hi[(size_t)i * n + k];
        if (!isfinite(l) || !isfinite(h)) bits |= 1u;
        if (l > h) bits |= 4u;
        if (!isfinite(y[(size_t)j * n + k])) bits |= 1u;
        double xm = v[3] > 0.0 ? -v[4] / (2.0 * v[3]) : (v[4] > 0.0 ? l : h);
        xm = clampd(xm, l, h);
        s0 += v[5];
        smin += v[3] * xm * xm + v[4] * xm + v[5];
    }
    s0 = warp_sum(s0);
    smin = warp_sum(smin);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s0;
        sh[1][threadIdx.x >> 5] = smin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        sumg0[pr] = a;
        if (isnan(c[i])) bits |= 16u;
        else if (b > c[i] * (1.0 + 1e-12) + 1e-12) bits |= 8u;
        scal[pr] = cold ? 0.0 : lam[pr];
        scal[mq + pr] = cold ? 0.0 : zeta[pr];
        scal[2 * mq + pr] = cold ? 0.0 : hh[pr];
        scal[3 * mq + pr] = cold ? 0.0 : pp[pr];
        scal[4 * mq + pr] = cold ? 0.0 : nu[pr];
        if (j == 0) scal[5 * mq + i] = cold ? 0.0 : x1[i];
        if (pr == 0) {
            double *tail = scal + 5 * mq + m;
            tail[0] = rho1;
            tail[1] = rho2;
            tail[2] = rho3;
            tail[3] = rho4;
            tail[4] = cold ? 1.0 : 0.0;
            tail[5] = 1.0;
            *bar = 0u;
            *status = 0;
        }
    }
    if (bits) atomicOr(flags, bits);
}

// The zero start of the element and column state (x = clamp(0), s = mu = 0),
// written only once the problem has passed validation.
__global__ void noalloc_cold_start(int n, int m, int q, const double *lo, const double *hi, double *x, double *s,
                                   double *mu)
{
    const int64_t ne = (int64_t)m * q * n, nc = (int64_t)q * n;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ne; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / n;
        const int k = (int)(t - r * n), i = (int)(r / q);
        x[t] = clampd(0.0, lo[(size_t)i * n + k], hi[(size_t)i * n + k]);
        if (t < nc) {
            s[t] = 0.0;
            mu[t] = 0.0;
        }
    }
}

// Copies the final scalar state back to the caller's arrays.
__global__ void noalloc_finish(int m, int q, const double *scal, double *lam, double *zeta, double *hh,
                               double *pp, double *nu, double *x1)
{
    const int mq = m * q;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < mq; t += gridDim.x * blockDim.x) {
        lam[t] = scal[t];
        zeta[t] = scal[mq + t];
        hh[t] = scal[2 * mq + t];
        pp[t] = scal[3 * mq + t];
        nu[t] = scal[4 * mq + t];
        if (t < m) x1[t] = scal[5 * mq + t];
    }
}

__global__ void noalloc_zero_flags(unsigned *flags) { *flags = 0u; }

// Device address of the scratch array for the current device (set-up on the
// first call per device).
admm_status scratch_for_current_device(double **out, int *dev_out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nfail(ADMM_ECUDA, "no usable current CUDA device");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return nfail(ADMM_ECUDA, "cudaGetSymbolAddress failed: ", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = (double *)g_scratch_ptr[dev];
    *dev_out = dev;
    return ADMM_OK;
}

} // namespace

extern "C" admm_status admm_solve_noalloc(const admm_problem *P, const admm_params *prm, admm_state *st,
                                          admm_result *out, void *stream)
{
    clear_last_error();
    if (!P || !prm || !st) return nfail(ADMM_EINVAL, "problem, params and state are required");
    if (!P->on_device || !st->on_device)
        return nfail(ADMM_EINVAL, "problem and state arrays must be device memory (on_device = 1)");
    if (P->n < 1 || P->m < 1 || P->q < 1) return nfail(ADMM_EINVAL, "n, m, q must be >= 1");
    if (P->coef_shared != 0) return nfail(ADMM_EUNSUPPORTED, "coef_shared is not available here");
    if (P->m > ADMM_MAX_M) return nfail(ADMM_EUNSUPPORTED, "m exceeds ADMM_MAX_M");
    if ((int64_t)P->m * P->q > ADMM_MAX_PAIRS) return nfail(ADMM_EUNSUPPORTED, "m*q exceeds ADMM_MAX_PAIRS");
    const double *arrs[] = {P->f2, P->f1, P->f0, P->g2, P->g1, P->g0, P->x_lo, P->x_hi, P->y, P->c,
                            st->x, st->s, st->mu, st->lam, st->zeta, st->h, st->p, st->nu, st->x1};
    for (const double *a : arrs)
        if (!a) return nfail(ADMM_EINVAL, "a problem or state array is NULL");
    for (int t = 0; t < 4; ++t)
        if (!(prm->rho[t] > 0.0) || !std::isfinite(prm->rho[t])) return nfail(ADMM_EINVAL, "rho must be finite and > 0");
    if (prm->max_iter < 1 || prm->check_every < 1) return nfail(ADMM_EINVAL, "max_iter and check_every must be >= 1");
    if (prm->precision != ADMM_FP64) return nfail(ADMM_EUNSUPPORTED, "only precision ADMM_FP64 is available here");
    if ((prm->xmin_mode != ADMM_XMIN_EXACT && prm->xmin_mode != ADMM_XMIN_PAPER) ||
        (prm->sweep != ADMM_GAUSS_SEIDEL && prm->sweep != ADMM_JACOBI) || (prm->adapt_rho && !(prm->tau > 1.0)) ||
        prm->adapt_start < 0)
        return nfail(ADMM_EINVAL, "bad xmin_mode, sweep, tau or adapt_start");

    double *scr = nullptr;
    int dev = -1;
    admm_status ss = scratch_for_current_device(&scr, &dev);
    if (ss != ADMM_OK) return ss;

    const int n = P->n, m = P->m, q = P->q, mq = m * q;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nfail(ADMM_ECUDA, "cudaDeviceGetAttribute failed");
    const size_t smem = single_smem_bytes(m, q, ADMM_FP64);
    // the same launch shape as admm_create
    const SingleShape sh = single_shape(prm->precision, m, q, n, nsm, smem);
    if (sh.grid < 1) return nfail(ADMM_EUNSUPPORTED, "solve kernel cannot be resident");
    const int64_t ncols = (int64_t)q * n, chunk = sh.chunk;
    const int grid = sh.grid, nbmax = sh.nbmax;
    // scratch layout (doubles, each region 32-double aligned)
    auto al = [](size_t v) { return (v + 31) / 32 * 32; };
    const size_t n_part = al((size_t)2 * q * nbmax * m * 4), n_cpart = al((size_t)2 * grid * 4);
    const size_t n_scal = al((size_t)scal_size(m, q)), n_sumg0 = al((size_t)mq), n_info = al(kInfo), n_words = 32;
    const size_t need = n_part + n_cpart + n_scal + n_sumg0 + n_info + n_words;
    if (need > kScratchDoubles) {
        char d[160];
        snprintf(d, sizeof d, " (needs %zu bytes, the fixed scratch holds %zu bytes)", need * 8, kScratchDoubles * 8);
        return nfail(ADMM_EUNSUPPORTED, "instance too large for the no-allocation scratch", d);
    }
    double *part = scr, *cpart = part + n_part, *scal = cpart + n_cpart, *sumg0 = scal + n_scal;
    double *info = sumg0 + n_sumg0;
    unsigned *words = (unsigned *)(info + n_info);
    unsigned *bar = words, *flags = words + 1;
    int *status = (int *)(words + 2);

    cudaStream_t cs = (cudaStream_t)stream;
    noalloc_zero_flags<<<1, 1, 0, cs>>>(flags);
    noalloc_prepare<<<mq, 256, 0, cs>>>(n, m, q, P->f2, P->f1, P->f0, P->g2, P->g1, P->g0, P->x_lo, P->x_hi, P->y,
                                       P->c, st->lam, st->zeta, st->h, st->p, st->nu, st->x1,
                                       st->cold ? prm->rho[0] : st->rho[0],
                                       st->cold ? (prm->rho2_over_n ? prm->rho[1] / (double)n : prm->rho[1]) : st->rho[1],
                                       st->cold ? prm->rho[2] : st->rho[2], st->cold ? prm->rho[3] : st->rho[3],
                                       st->cold ? 1 : 0, scal, sumg0, bar, status, flags);
    cudaError_t e = cudaGetLastError();
    unsigned hflags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return nfail(ADMM_ECUDA, "prepare: ", cudaGetErrorString(e));
    if (hflags) {
        std::string why;
        if (hflags & 1u) why += " non-finite data;";
        if (hflags & 2u) why += " f2 < 0 or g2 < 0;";
        if (hflags & 4u) why += " x_lo > x_hi;";
        if (hflags & 16u) why += " c is NaN;";
        if (hflags & 8u) why += " sum_k min g > c (infeasible);";
        return nfail(ADMM_EINVAL, "invalid problem:", why.c_str());
    }
    if (st->cold) {
        const int64_t ne = (int64_t)mq * n;
        const int blocks = (int)std::min<int64_t>((ne + 255) / 256, (int64_t)nsm * 8);
        noalloc_cold_start<<<blocks, 256, 0, cs>>>(n, m, q, P->x_lo, P->x_hi, st->x, st->s, st->mu);
        if ((e = cudaGetLastError()) != cudaSuccess) return nfail(ADMM_ECUDA, "cold start: ", cudaGetErrorString(e));
    }

    SingleArgs a{};
    a.n = n;
    a.m = m;
    a.q = q;
    a.ld = n;
    a.rs = n;
    a.ncols = ncols;
    a.chunk = chunk;
    a.pieces = sh.pieces;
    a.cq = q;
    a.cj = 1;
    a.nbmax = nbmax;
    a.grid = grid;
    a.f2 = P->f2;
    a.f1 = P->f1;
    a.f0 = P->f0;
    a.g2 = P->g2;
    a.g1 = P->g1;
    a.g0 = P->g0;
    a.lo = P->x_lo;
    a.hi = P->x_hi;
    a.y = P->y;
    a.c = P->c;
    a.sumg0 = sumg0;
    a.x = st->x;
    a.s = st->s;
    a.mu = st->mu;
    a.scal = scal;
    a.part = part;
    a.cpart = cpart;
    a.bar = bar;
    a.status = status;
    a.info = info;
    a.r_tol = prm->r_tol;
    a.s_tol = prm->s_tol;
    a.adapt_target = prm->r_tol / prm->s_tol;
    a.adapt_start = prm->adapt_start;
    a.tau = prm->tau;
    a.max_iter = prm->max_iter;
    a.check_every = prm->check_every;
    a.xmin_mode = prm->xmin_mode;
    a.sweep = prm->sweep;
    a.adapt = prm->adapt_rho;
    a.spin_ns = 2000000000LL;
    e = launch_single(prm->precision, sh.minb, a, smem, cs);
    if (e != cudaSuccess) return nfail(ADMM_ECUDA, "solve launch: ", cudaGetErrorString(e));
    noalloc_finish<<<(mq + 255) / 256, 256, 0, cs>>>(m, q, scal, st->lam, st->zeta, st->h, st->p, st->nu, st->x1);
    double hinfo[kInfo], tail[6];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tail, scal + 5 * mq + m, sizeof tail, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && out && out->x)
        e = cudaMemcpyAsync(out->x, st->x, sizeof(double) * (size_t)mq * n,
                            out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && out && out->x1)
        e = cudaMemcpyAsync(out->x1, st->x1, sizeof(double) * m,
                            out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return nfail(ADMM_ECUDA, "solve: ", cudaGetErrorString(e));
    for (int t = 0; t < 4; ++t) st->rho[t] = tail[t];
    st->cold = tail[4] != 0.0;
    admm_status s = ADMM_OK;
    if (hinfo[12] != 0.0) s = (admm_status)(int)hinfo[12];
    else if (hinfo[1] == 0.0) s = ADMM_ENOTCONVERGED;
    if (out) {
        out->iters = (int32_t)hinfo[0];
        out->converged = hinfo[1] != 0.0;
        out->r = hinfo[2];
        out->sigma = hinfo[3];
        out->objective = hinfo[11];
        out->status = s;
    }
    if (s == ADMM_ETIMEOUT) return nfail(s, "a grid barrier wait timed out");
    return s;
}

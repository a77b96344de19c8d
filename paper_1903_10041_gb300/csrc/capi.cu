// Host side of the C ABI declared in include/admm.h: validation, device
// layout, launch configuration and state import/export for the
// single-instance solver.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

using namespace admm_impl;

namespace {

thread_local std::string g_err;

admm_status fail(admm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(call)                                                                                     \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                       \
    } while (0)

// Element validation flags (bits)
enum : unsigned {
    V_NONFINITE = 1u,   // a coefficient, bound or demand is NaN or infinite
    V_NONCONVEX = 2u,   // f2 < 0 or g2 < 0 (Assumption 1)
    V_BOUNDS = 4u,      // x_lo > x_hi
    V_INFEASIBLE = 8u,  // sum_k min g > c for some (i, j)
    V_CNAN = 16u        // c is NaN
};

__global__ void validate_elements(int n, int m, int q, int ld, int cq, int cj, const double *f2, const double *f1,
                                  const double *f0, const double *g2, const double *g1, const double *g0,
                                  const double *lo, const double *hi, const double *y, unsigned *flags)
{
    const int64_t total = (int64_t)m * q * n;
    unsigned bits = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % n);
        const int64_t r = t / n; // i*q + j
        const int i = (int)(r / q), j = (int)(r % q);
        const size_t e = ((size_t)i * cq + (size_t)j * cj) * ld + k; // coefficient row of (i, j)
        const double v[6] = {f2[e], f1[e], f0[e], g2[e], g1[e], g0[e]};
        for (int u = 0; u < 6; ++u)
            if (!isfinite(v[u])) bits |= V_NONFINITE;
        if (v[0] < 0.0 || v[3] < 0.0) bits |= V_NONCONVEX;
        if (j == 0) {
            const double a = lo[(size_t)i * ld + k], b = hi[(size_t)i * ld + k];
            if (!isfinite(a) || !isfinite(b)) bits |= V_NONFINITE;
            if (a > b) bits |= V_BOUNDS;
        }
        if (i == 0 && !isfinite(y[(size_t)j * ld + k])) bits |= V_NONFINITE;
    }
    if (bits) atomicOr(flags, bits);
}

// One CTA per pair (i, j): sum_k beta_0 (kept for the solve) and the
// smallest achievable sum_k g (for the sure-infeasibility check).
__global__ void pair_sums(int n, int m, int q, int ld, int cq, int cj, const double *g2, const double *g1,
                          const double *g0, const double *lo, const double *hi, const double *c, double *sumg0,
                          unsigned *flags)
{
    __shared__ double sh[2][32];
    const int pr = blockIdx.x, i = pr / q;
    const size_t base = ((size_t)i * cq + (size_t)(pr - i * q) * cj) * ld;
    double s0 = 0.0, smin = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double a2 = g2[base + k], a1 = g1[base + k], a0 = g0[base + k];
        const double l = lo[(size_t)i * ld + k], h = hi[(size_t)i * ld + k];
        double xm = a2 > 0.0 ? -a1 / (2.0 * a2) : (a1 > 0.0 ? l : h);
        xm = clampd(xm, l, h);
        s0 += a0;
        smin += a2 * xm * xm + a1 * xm + a0;
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
        const double ci = c[i];
        if (isnan(ci)) atomicOr(flags, V_CNAN);
        else if (b > ci * (1.0 + 1e-12) + 1e-12) atomicOr(flags, V_INFEASIBLE);
    }
}

__global__ void selftest_barrier_kernel(unsigned *bar, int *status, long long spin_ns, unsigned extra)
{
    // Waits for `extra` more arrivals than the grid can provide.
    grid_barrier(bar, gridDim.x + extra, status, spin_ns, ADMM_ETIMEOUT);
}

bool params_ok(const admm_params *p)
{
    if (!p) return !fail(ADMM_EINVAL, "params is NULL");
    for (int t = 0; t < 4; ++t)
        if (!(p->rho[t] > 0.0) || !std::isfinite(p->rho[t]))
            return !fail(ADMM_EINVAL, "rho[%d] = %g must be finite and > 0", t, p->rho[t]);
    if (!(p->r_tol >= 0.0) || !(p->s_tol >= 0.0)) return !fail(ADMM_EINVAL, "r_tol and s_tol must be >= 0");
    if (p->max_iter < 1) return !fail(ADMM_EINVAL, "max_iter must be >= 1");
    if (p->check_every < 1) return !fail(ADMM_EINVAL, "check_every must be >= 1");
    if (p->precision != ADMM_FP64 && p->precision != ADMM_MIXED && p->precision != ADMM_MIXED_FP64CUBIC)
        return !fail(ADMM_EINVAL, "bad precision %d", p->precision);
    if (p->xmin_mode != ADMM_XMIN_EXACT && p->xmin_mode != ADMM_XMIN_PAPER)
        return !fail(ADMM_EINVAL, "bad xmin_mode %d", p->xmin_mode);
    if (p->sweep != ADMM_GAUSS_SEIDEL && p->sweep != ADMM_JACOBI) return !fail(ADMM_EINVAL, "bad sweep %d", p->sweep);
    if (p->adapt_rho && !(p->tau > 1.0)) return !fail(ADMM_EINVAL, "tau must be > 1 with adapt_rho");
    if (p->adapt_start < 0) return !fail(ADMM_EINVAL, "adapt_start must be >= 0");
    for (int t = 0; t < 2; ++t)
        if (p->reserved[t]) return !fail(ADMM_EINVAL, "reserved fields must be 0");
    return true;
}

long long spin_limit_ns()
{
    const char *e = getenv("ADMM_SPIN_NS");
    long long v = e ? atoll(e) : 0;
    return v > 0 ? v : 2000000000LL; // 2 s per barrier wait
}

} // namespace

namespace admm_impl {
void set_last_error(const char *msg) { g_err = msg; }
void clear_last_error() { g_err.clear(); }
} // namespace admm_impl

struct admm_handle {
    int n = 0, m = 0, q = 0, ld = 0, dev = 0, nsm = 0;
    admm_params prm{};
    int esz = 8;                 // bytes per stored value: 8 (FP64) or 4 (mixed)
    // problem, padded rows of ld, storage type by esz
    void *f2 = nullptr, *f1 = nullptr, *f0 = nullptr, *g2 = nullptr, *g1 = nullptr, *g0 = nullptr;
    void *lo = nullptr, *hi = nullptr, *y = nullptr;
    double *c = nullptr, *sumg0 = nullptr;
    // state
    void *x = nullptr, *s = nullptr, *mu = nullptr;
    void *s_lo = nullptr, *mu_lo = nullptr; // mixed: low parts of float-float s, mu (inside s, mu allocations)
    double *scal = nullptr;
    // scratch
    double *part = nullptr, *cpart = nullptr, *info = nullptr;
    double *tmp64 = nullptr;     // FP64 staging for mixed-precision import/export (lazy)
    size_t tmp64_n = 0;
    unsigned *bar = nullptr, *flags = nullptr;
    int *status = nullptr;
    double *info_host = nullptr; // pinned
    cudaEvent_t done = nullptr;  // recorded after each queued solve (admm_wait)
    // launch shape
    int grid = 0, nbmax = 0, rs = 0, minb = 1;
    int64_t chunk = 0, ncols = 0;
    int pieces = 0;
    size_t smem = 0;
    int cshared = 0; // coefficients shared by the scenarios ([m][ld])
};

namespace {

// Host-side fault injection for the failure paths of admm_create: with the
// environment variable ADMM_FAULT_ALLOC = k (k >= 1), the k-th device
// allocation of each admm_create call reports cudaErrorMemoryAllocation
// instead of allocating.  Unset (the normal case) it costs one getenv.
struct AllocFault {
    long long fail_at = 0, count = 0;
    AllocFault()
    {
        const char *v = std::getenv("ADMM_FAULT_ALLOC");
        fail_at = v ? std::atoll(v) : 0;
    }
};

template <class T> cudaError_t dev_malloc(AllocFault &af, T **p, size_t bytes)
{
    if (af.fail_at > 0 && ++af.count == af.fail_at) return cudaErrorMemoryAllocation;
    return cudaMalloc((void **)p, bytes);
}

template <class T> void dfree(T *&p)
{
    if (p) cudaFree((void *)p);
    p = nullptr;
}

void free_all(admm_handle *h)
{
    void **vp[] = {&h->f2, &h->f1, &h->f0, &h->g2, &h->g1, &h->g0, &h->lo, &h->hi, &h->y, &h->x, &h->s, &h->mu};
    for (void **p : vp) dfree(*p);
    dfree(h->c);
    dfree(h->sumg0);
    dfree(h->scal);
    dfree(h->part);
    dfree(h->cpart);
    dfree(h->info);
    dfree(h->tmp64);
    dfree(h->bar);
    dfree(h->flags);
    dfree(h->status);
    if (h->info_host) cudaFreeHost(h->info_host);
    h->info_host = nullptr;
    if (h->done) cudaEventDestroy(h->done);
    h->done = nullptr;
}

#ifdef ADMM_DEBUG_BOUNDS
// Self-test of the bounds check: index 20 of a 16-float buffer is recorded
// and redirected to 0 (the access stays inside the buffer).
__global__ void bounds_selftest_kernel(float *buf, unsigned long long *rec)
{
    if (threadIdx.x == 0) {
        const size_t k = ADMM_IDX((size_t)20, 1, (size_t)16, rec, DBG_SELFTEST);
        buf[k] += 1.0f;
    }
}
#endif

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// rows x n doubles from a (host or device) dense source into a padded device array
cudaError_t put_rows(double *dst, int ld, const double *src, int n, int64_t rows, bool src_dev)
{
    return cudaMemcpy2D(dst, (size_t)ld * 8, src, (size_t)n * 8, (size_t)n * 8, (size_t)rows,
                        src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
}

cudaError_t ensure_tmp(admm_handle *h, size_t count)
{
    if (h->tmp64_n >= count) return cudaSuccess;
    dfree(h->tmp64);
    h->tmp64_n = 0;
    cudaError_t e = cudaMalloc(&h->tmp64, count * 8);
    if (e == cudaSuccess) h->tmp64_n = count;
    return e;
}

// Handle array (padded, storage type; `lo` = low parts of a float-float
// array or NULL) -> caller's dense FP64 rows.
cudaError_t export_rows(admm_handle *h, double *dst, bool dst_dev, const void *src, int64_t rows, cudaStream_t st,
                        const void *lo = nullptr)
{
    const int n = h->n, ld = h->ld;
    const cudaMemcpyKind k = dst_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (h->esz == 8)
        return cudaMemcpy2DAsync(dst, (size_t)n * 8, src, (size_t)ld * 8, (size_t)n * 8, (size_t)rows, k, st);
    double *to = dst;
    if (!dst_dev) {
        cudaError_t e = ensure_tmp(h, (size_t)rows * n);
        if (e != cudaSuccess) return e;
        to = h->tmp64;
    }
    if (lo) convert_rows_ff_to_f64(to, n, (const float *)src, (const float *)lo, ld, n, rows, st);
    else convert_rows_f32_to_f64(to, n, (const float *)src, ld, n, rows, st);
    if (dst_dev) return cudaGetLastError();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(dst, h->tmp64, (size_t)rows * n * 8, k, st);
}

// Caller's dense FP64 rows -> handle array (padded, storage type; `lo` as in export_rows).
cudaError_t import_rows(admm_handle *h, void *dst, const double *src, bool src_dev, int64_t rows, cudaStream_t st,
                        void *lo = nullptr)
{
    const int n = h->n, ld = h->ld;
    const cudaMemcpyKind k = src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (h->esz == 8)
        return cudaMemcpy2DAsync(dst, (size_t)ld * 8, src, (size_t)n * 8, (size_t)n * 8, (size_t)rows, k, st);
    const double *from = src;
    if (!src_dev) {
        cudaError_t e = ensure_tmp(h, (size_t)rows * n);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(h->tmp64, src, (size_t)rows * n * 8, k, st);
        if (e != cudaSuccess) return e;
        from = h->tmp64;
    }
    if (lo) split_rows_f64_to_ff((float *)dst, (float *)lo, ld, from, n, n, rows, st);
    else convert_rows_f64_to_f32((float *)dst, ld, from, n, n, rows, st);
    return cudaGetLastError();
}

template <class T>
__global__ void init_x_t(int n, int m, int q, int ld, const T *lo, const T *hi, T *x)
{
    const int64_t total = (int64_t)m * q * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t % n);
        const int64_t r = t / n;
        const int i = (int)(r / q);
        const T l = lo[(size_t)i * ld + k], u = hi[(size_t)i * ld + k];
        x[(size_t)r * ld + k] = (T)0 < l ? l : ((T)0 > u ? u : (T)0);
    }
}

admm_status reset_state(admm_handle *h)
{
    const int m = h->m, q = h->q, mq = m * q;
    const int g = std::max(1, std::min(h->nsm * 4, (int)((int64_t)m * q * h->n / 256 + 1)));
    if (h->esz == 8)
        init_x_t<double><<<g, 256>>>(h->n, m, q, h->ld, (const double *)h->lo, (const double *)h->hi, (double *)h->x);
    else
        init_x_t<float><<<g, 256>>>(h->n, m, q, h->ld, (const float *)h->lo, (const float *)h->hi, (float *)h->x);
    CUDA_TRY(cudaGetLastError());
    const size_t cb = (size_t)8 * q * h->ld; // FP64, or float-float hi + lo rows
    CUDA_TRY(cudaMemset(h->s, 0, cb));
    CUDA_TRY(cudaMemset(h->mu, 0, cb));
    std::vector<double> sc(scal_size(m, q), 0.0);
    for (int t = 0; t < 4; ++t) sc[5 * mq + m + t] = h->prm.rho[t];
    if (h->prm.rho2_over_n) sc[5 * mq + m + 1] = h->prm.rho[1] / (double)h->n;
    sc[5 * mq + m + 4] = 1.0; // cold
    sc[5 * mq + m + 5] = 1.0; // no pending mu rescale
    CUDA_TRY(cudaMemcpy(h->scal, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaDeviceSynchronize());
    return ADMM_OK;
}

} // namespace

extern "C" {

void admm_default_params(admm_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    for (int t = 0; t < 4; ++t) p->rho[t] = 1.0;
    p->r_tol = 1e-6;
    p->s_tol = 1e-6;
    p->tau = 1.1;
    p->max_iter = 5000;
    p->check_every = 10;
    p->precision = ADMM_FP64;
    p->xmin_mode = ADMM_XMIN_EXACT;
    p->sweep = ADMM_GAUSS_SEIDEL;
    p->adapt_rho = 0;
}

const char *admm_last_error(void) { return g_err.c_str(); }

const char *admm_status_string(admm_status s)
{
    switch (s) {
    case ADMM_OK: return "ok";
    case ADMM_EINVAL: return "invalid argument";
    case ADMM_ENOMEM: return "out of memory";
    case ADMM_ECUDA: return "CUDA error";
    case ADMM_ETIMEOUT: return "device wait timed out";
    case ADMM_ENOTCONVERGED: return "not converged";
    case ADMM_EUNSUPPORTED: return "unsupported size or mode";
    case ADMM_EPENDING: return "pending";
    case ADMM_ECANCELLED: return "cancelled";
    case ADMM_EBOUNDS: return "element access out of bounds (checked build)";
    }
    return "unknown status";
}

admm_status admm_create(const admm_problem *P, const admm_params *prm, admm_handle **out)
{
    TraceRange trace_("admm_create");
    g_err.clear();
    if (!out) return fail(ADMM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!P) return fail(ADMM_EINVAL, "problem is NULL");
    if (P->n < 1 || P->m < 1 || P->q < 1) return fail(ADMM_EINVAL, "n, m, q must be >= 1 (got %d, %d, %d)", P->n, P->m, P->q);
    if (P->m > ADMM_MAX_M) return fail(ADMM_EUNSUPPORTED, "m = %d exceeds ADMM_MAX_M = %d", P->m, ADMM_MAX_M);
    if ((int64_t)P->m * P->q > ADMM_MAX_PAIRS)
        return fail(ADMM_EUNSUPPORTED, "m*q = %lld exceeds ADMM_MAX_PAIRS = %d", (long long)P->m * P->q, ADMM_MAX_PAIRS);
    const double *arrs[] = {P->f2, P->f1, P->f0, P->g2, P->g1, P->g0, P->x_lo, P->x_hi, P->y, P->c};
    for (const double *a : arrs)
        if (!a) return fail(ADMM_EINVAL, "a problem array is NULL");
    if (P->coef_shared != 0 && P->coef_shared != 1) return fail(ADMM_EINVAL, "coef_shared must be 0 or 1");
    if (!params_ok(prm)) return g_err.find("precision") != std::string::npos ? ADMM_EUNSUPPORTED : ADMM_EINVAL;

    admm_handle *h = new admm_handle();
    AllocFault af;
    const bool mixed = prm->precision != ADMM_FP64;
    h->cshared = P->coef_shared;
    h->n = P->n;
    h->m = P->m;
    h->q = P->q;
    h->esz = mixed ? 4 : 8;
    h->ld = mixed ? (P->n + 63) / 64 * 64 : (P->n + 31) / 32 * 32;
    h->prm = *prm;
    admm_status st = ADMM_OK;
    // FP64 staging copies of the problem (the final arrays in FP64 mode)
    double *s64[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    auto bail = [&](admm_status s) {
        for (double *&p : s64) dfree(p); // staging copies not yet owned by the handle
        free_all(h);
        delete h;
        return s;
    };
#define TRY(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA, "%s: %s", #call,    \
                             cudaGetErrorString(e_)));                                                     \
    } while (0)
    TRY(cudaGetDevice(&h->dev));
    TRY(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
    const int n = h->n, m = h->m, q = h->q, ld = h->ld, mq = m * q;
    const int crow = h->cshared ? m : mq; // coefficient rows
    const size_t ne = (size_t)mq * ld, nf = (size_t)crow * ld, nb = (size_t)m * ld, nc = (size_t)q * ld;
    const size_t cnt[9] = {nf, nf, nf, nf, nf, nf, nb, nb, nc};
    for (int t = 0; t < 9; ++t) {
        TRY(dev_malloc(af, &s64[t], cnt[t] * 8));
        TRY(cudaMemset(s64[t], 0, cnt[t] * 8));
    }
    TRY(dev_malloc(af, &h->c, m * 8));
    TRY(dev_malloc(af, &h->sumg0, mq * 8));
    TRY(dev_malloc(af, &h->scal, scal_size(m, q) * 8));
    TRY(dev_malloc(af, &h->info, kInfo * 8));
    TRY(dev_malloc(af, &h->bar, sizeof(unsigned)));
    TRY(dev_malloc(af, &h->flags, sizeof(unsigned)));
    TRY(dev_malloc(af, &h->status, sizeof(int)));
    TRY(cudaMallocHost(&h->info_host, kInfo * 8));
    for (int t = 0; t < kInfo; ++t) h->info_host[t] = 0.0;
    TRY(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));

    const bool dev = P->on_device != 0;
    const double *src[9] = {P->f2, P->f1, P->f0, P->g2, P->g1, P->g0, P->x_lo, P->x_hi, P->y};
    const int64_t rows[9] = {crow, crow, crow, crow, crow, crow, m, m, q};
    for (int t = 0; t < 9; ++t) TRY(put_rows(s64[t], ld, src[t], n, rows[t], dev));
    TRY(cudaMemcpy(h->c, P->c, m * 8, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));

    // validation (Assumptions 1 and 3, bounds, sure infeasibility)
    TRY(cudaMemset(h->flags, 0, sizeof(unsigned)));
    const int cq = h->cshared ? 1 : q, cj = h->cshared ? 0 : 1;
    validate_elements<<<std::max(1, std::min(h->nsm * 8, (int)(ne / 256 + 1))), 256>>>(
        n, m, q, ld, cq, cj, s64[0], s64[1], s64[2], s64[3], s64[4], s64[5], s64[6], s64[7], s64[8], h->flags);
    TRY(cudaGetLastError());
    pair_sums<<<mq, 256>>>(n, m, q, ld, cq, cj, s64[3], s64[4], s64[5], s64[6], s64[7], h->c, h->sumg0,
                           h->flags);
    TRY(cudaGetLastError());
    unsigned flags = 0;
    TRY(cudaMemcpy(&flags, h->flags, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags) {
        std::string why;
        if (flags & V_NONFINITE) why += " non-finite coefficient, bound or demand;";
        if (flags & V_NONCONVEX) why += " f2 < 0 or g2 < 0 (Assumption 1 needs convex f, g);";
        if (flags & V_BOUNDS) why += " x_lo > x_hi;";
        if (flags & V_CNAN) why += " c is NaN;";
        if (flags & V_INFEASIBLE) why += " sum_k min g > c for some (i, j): infeasible;";
        return bail(fail(ADMM_EINVAL, "invalid problem:%s", why.c_str()));
    }
    void **dst[9] = {&h->f2, &h->f1, &h->f0, &h->g2, &h->g1, &h->g0, &h->lo, &h->hi, &h->y};
    if (!mixed) {
        for (int t = 0; t < 9; ++t) {
            *dst[t] = s64[t];
            s64[t] = nullptr;
        }
        TRY(dev_malloc(af, &h->x, ne * 8));
        TRY(dev_malloc(af, &h->s, nc * 8));
        TRY(dev_malloc(af, &h->mu, nc * 8));
    } else {
        for (int t = 0; t < 9; ++t) {
            TRY(dev_malloc(af, dst[t], cnt[t] * 4));
            convert_rows_f64_to_f32((float *)*dst[t], ld, s64[t], ld, ld, rows[t], 0);
            TRY(cudaGetLastError());
        }
        TRY(cudaDeviceSynchronize());
        for (double *&p : s64) dfree(p);
        TRY(dev_malloc(af, &h->x, ne * 4));
        TRY(dev_malloc(af, &h->s, nc * 8));   // float-float: hi rows then lo rows
        TRY(dev_malloc(af, &h->mu, nc * 8));
        h->s_lo = (float *)h->s + nc;
        h->mu_lo = (float *)h->mu + nc;
        TRY(cudaMemset(h->x, 0, ne * 4));
    }

    // launch shape: contiguous equal column chunks, all SMs busy
    h->smem = single_smem_bytes(m, q, prm->precision);
    h->rs = mixed ? ld : n;
    h->ncols = (int64_t)q * h->rs;
    const SingleShape sh = single_shape(prm->precision, m, q, h->rs, h->nsm, h->smem);
    if (sh.grid < 1) return bail(fail(ADMM_EUNSUPPORTED, "solve kernel cannot be resident (smem %zu B)", h->smem));
    h->chunk = sh.chunk;
    h->pieces = sh.pieces;
    h->grid = sh.grid;
    h->nbmax = sh.nbmax;
    h->minb = sh.minb;
    TRY(dev_malloc(af, &h->part, sizeof(double) * 2 * (size_t)q * h->nbmax * m * 4));
    TRY(dev_malloc(af, &h->cpart, sizeof(double) * 2 * (size_t)h->grid * 4));
    st = reset_state(h);
    if (st != ADMM_OK) return bail(st);
#undef TRY
    *out = h;
    return ADMM_OK;
}

admm_status admm_set_params(admm_handle *h, const admm_params *prm)
{
    g_err.clear();
    if (!h) return fail(ADMM_EINVAL, "handle is NULL");
    if (!params_ok(prm)) return g_err.find("precision") != std::string::npos ? ADMM_EUNSUPPORTED : ADMM_EINVAL;
    if ((prm->precision == ADMM_FP64) != (h->prm.precision == ADMM_FP64))
        return fail(ADMM_EINVAL, "the storage precision (FP64 or mixed) is fixed at admm_create");
    DeviceGuard dg(h->dev);
    h->prm = *prm;
    const int mq = h->m * h->q;
    double rho[4] = {prm->rho[0], prm->rho[1], prm->rho[2], prm->rho[3]};
    if (prm->rho2_over_n) rho[1] /= (double)h->n;
    CUDA_TRY(cudaMemcpy(h->scal + 5 * mq + h->m, rho, 4 * 8, cudaMemcpyHostToDevice));
    return ADMM_OK;
}

admm_status admm_reset(admm_handle *h)
{
    g_err.clear();
    if (!h) return fail(ADMM_EINVAL, "handle is NULL");
    DeviceGuard dg(h->dev);
    return reset_state(h);
}

// Status of a finished solve from its info record ([15]: the bounds record
// of checked builds, as raw bits).
static admm_status result_status(const double *inf)
{
    unsigned long long rec;
    std::memcpy(&rec, inf + 15, sizeof rec);
    if (rec != 0) return ADMM_EBOUNDS;
    if (inf[12] != 0.0) return (admm_status)(int)inf[12];
    return inf[1] == 0.0 ? ADMM_ENOTCONVERGED : ADMM_OK;
}

static void fill_result(const double *inf, admm_result *out)
{
    out->iters = (int32_t)inf[0];
    out->converged = inf[1] != 0.0;
    out->r = inf[2];
    out->sigma = inf[3];
    out->objective = inf[11];
    out->status = result_status(inf);
}

// Host function queued behind a solve: copies its record into the caller's
// admm_result (no CUDA calls in here).
struct ResultFill {
    const double *info_host;
    admm_result *out;
};
static void CUDART_CB fill_result_cb(void *p)
{
    ResultFill *rf = (ResultFill *)p;
    fill_result(rf->info_host, rf->out);
    delete rf;
}

static admm_status load_state(admm_handle *h, const admm_state *w, cudaStream_t st)
{
    const int m = h->m, q = h->q, mq = m * q;
    const bool dev = w->on_device != 0;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!w->x || !w->s || !w->mu || !w->lam || !w->zeta || !w->h || !w->p || !w->nu || !w->x1)
        return fail(ADMM_EINVAL, "warm state has a NULL array");
    for (int t = 0; t < 4; ++t)
        if (!(w->rho[t] > 0.0)) return fail(ADMM_EINVAL, "warm state rho[%d] must be > 0", t);
    CUDA_TRY(import_rows(h, h->x, w->x, dev, mq, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(import_rows(h, h->s, w->s, dev, q, st, h->s_lo));
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(import_rows(h, h->mu, w->mu, dev, q, st, h->mu_lo));
    const double *pairs[5] = {w->lam, w->zeta, w->h, w->p, w->nu};
    for (int t = 0; t < 5; ++t) CUDA_TRY(cudaMemcpyAsync(h->scal + (size_t)t * mq, pairs[t], mq * 8, k, st));
    CUDA_TRY(cudaMemcpyAsync(h->scal + 5 * mq, w->x1, m * 8, k, st));
    double tail[6] = {w->rho[0], w->rho[1], w->rho[2], w->rho[3], w->cold ? 1.0 : 0.0, 1.0};
    CUDA_TRY(cudaStreamSynchronize(st));
    CUDA_TRY(cudaMemcpy(h->scal + 5 * mq + m, tail, sizeof tail, cudaMemcpyHostToDevice));
    return ADMM_OK;
}

admm_status admm_solve(admm_handle *h, const admm_state *warm, admm_result *out, void *stream)
{
    TraceRange trace_("admm_solve");
    g_err.clear();
    if (!h) return fail(ADMM_EINVAL, "handle is NULL");
    DeviceGuard dg(h->dev);
    cudaStream_t st = (cudaStream_t)stream;
    if (warm) {
        admm_status s = load_state(h, warm, st);
        if (s != ADMM_OK) return s;
    }
    SingleArgs a{};
    a.n = h->n;
    a.m = h->m;
    a.q = h->q;
    a.ld = h->ld;
    a.rs = h->rs;
    a.ncols = h->ncols;
    a.chunk = h->chunk;
    a.pieces = h->pieces;
    a.cq = h->cshared ? 1 : h->q;
    a.cj = h->cshared ? 0 : 1;
    a.nbmax = h->nbmax;
    a.grid = h->grid;
    a.f2 = h->f2;
    a.f1 = h->f1;
    a.f0 = h->f0;
    a.g2 = h->g2;
    a.g1 = h->g1;
    a.g0 = h->g0;
    a.lo = h->lo;
    a.hi = h->hi;
    a.y = h->y;
    a.c = h->c;
    a.sumg0 = h->sumg0;
    a.x = h->x;
    a.s = h->s;
    a.mu = h->mu;
    a.s_lo = h->s_lo;
    a.mu_lo = h->mu_lo;
    a.scal = h->scal;
    a.part = h->part;
    a.cpart = h->cpart;
    a.bar = h->bar;
    a.status = h->status;
    a.info = h->info;
    a.r_tol = stop_r_tol(h->prm.precision, h->prm.r_tol);
    a.s_tol = stop_s_tol(h->prm.precision, h->prm.s_tol);
    a.adapt_target = h->prm.r_tol / h->prm.s_tol;
    a.adapt_start = h->prm.adapt_start;
    a.tau = h->prm.tau;
    a.max_iter = h->prm.max_iter;
    a.check_every = h->prm.check_every;
    a.xmin_mode = h->prm.xmin_mode;
    a.sweep = h->prm.sweep;
    a.adapt = h->prm.adapt_rho;
    a.spin_ns = spin_limit_ns();
    CUDA_TRY(cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
    CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CUDA_TRY(cudaMemsetAsync(h->info + 15, 0, sizeof(double), st));
    a.dbg = (unsigned long long *)(h->info + 15);
    CUDA_TRY(launch_single(h->prm.precision, h->minb, a, h->smem, st));
    CUDA_TRY(cudaMemcpyAsync(h->info_host, h->info, kInfo * 8, cudaMemcpyDeviceToHost, st));
    if (out && out->x) CUDA_TRY(export_rows(h, out->x, out->on_device != 0, h->x, (int64_t)h->m * h->q, st));
    if (out && out->x1)
        CUDA_TRY(cudaMemcpyAsync(out->x1, h->scal + 5 * h->m * h->q, h->m * 8,
                                 out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    if (out) {
        // fills *out when the stream reaches this point (valid after a sync)
        ResultFill *rf = new ResultFill{h->info_host, out};
        cudaError_t e = cudaLaunchHostFunc(st, fill_result_cb, rf);
        if (e != cudaSuccess) {
            delete rf;
            return fail(ADMM_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
        }
    }
    CUDA_TRY(cudaEventRecord(h->done, st));
    return ADMM_OK;
}

admm_status admm_wait(admm_handle *h, admm_result *out)
{
    g_err.clear();
    if (!h) return fail(ADMM_EINVAL, "handle is NULL");
    DeviceGuard dg(h->dev);
    CUDA_TRY(cudaEventSynchronize(h->done));
    if (out) fill_result(h->info_host, out);
    const admm_status s = result_status(h->info_host);
    if (s == ADMM_ETIMEOUT) return fail(s, "a grid barrier wait timed out");
    if (s == ADMM_EBOUNDS) {
        unsigned long long rec;
        std::memcpy(&rec, h->info_host + 15, sizeof rec);
        return fail(s, "element access out of bounds: array %d, index %lld", (int)(rec >> 56) - 1,
                    (long long)(rec & 0x00FFFFFFFFFFFFFFull));
    }
    if (s == ADMM_ENOTCONVERGED) g_err = "max_iter reached before the stop test passed";
    return s;
}

admm_status admm_get_state(admm_handle *h, admm_state *o, void *stream)
{
    g_err.clear();
    if (!h || !o) return fail(ADMM_EINVAL, "NULL argument");
    DeviceGuard dg(h->dev);
    cudaStream_t st = (cudaStream_t)stream;
    const int m = h->m, q = h->q, mq = m * q;
    const bool dev = o->on_device != 0;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (o->x) {
        CUDA_TRY(export_rows(h, o->x, dev, h->x, mq, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (o->s) {
        CUDA_TRY(export_rows(h, o->s, dev, h->s, q, st, h->s_lo));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    if (o->mu) {
        CUDA_TRY(export_rows(h, o->mu, dev, h->mu, q, st, h->mu_lo));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    double *pairs[5] = {o->lam, o->zeta, o->h, o->p, o->nu};
    for (int t = 0; t < 5; ++t)
        if (pairs[t]) CUDA_TRY(cudaMemcpyAsync(pairs[t], h->scal + (size_t)t * mq, mq * 8, k, st));
    if (o->x1) CUDA_TRY(cudaMemcpyAsync(o->x1, h->scal + 5 * mq, m * 8, k, st));
    double tail[6];
    CUDA_TRY(cudaMemcpyAsync(tail, h->scal + 5 * mq + m, sizeof tail, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int t = 0; t < 4; ++t) o->rho[t] = tail[t];
    o->cold = tail[4] != 0.0;
    return ADMM_OK;
}

admm_status admm_get_info(admm_handle *h, double *info_out, int count)
{
    g_err.clear();
    if (!h || !info_out || count < 1) return fail(ADMM_EINVAL, "NULL argument");
    for (int t = 0; t < count && t < kInfo; ++t) info_out[t] = h->info_host[t];
    return ADMM_OK;
}

admm_status admm_destroy(admm_handle *h)
{
    if (!h) return ADMM_OK;
    {
        DeviceGuard dg(h->dev);
        free_all(h);
    }
    delete h;
    return ADMM_OK;
}

admm_status admm_selftest_bounds(int *status_out, long long *index_out)
{
    g_err.clear();
    if (!status_out || !index_out) return fail(ADMM_EINVAL, "NULL argument");
#ifdef ADMM_DEBUG_BOUNDS
    float *buf = nullptr;
    unsigned long long *rec = nullptr;
    CUDA_TRY(cudaMalloc(&buf, 16 * sizeof(float) + sizeof(unsigned long long)));
    rec = (unsigned long long *)(buf + 16);
    cudaError_t e = cudaMemset(buf, 0, 16 * sizeof(float) + sizeof(unsigned long long));
    if (e == cudaSuccess) {
        bounds_selftest_kernel<<<1, 32>>>(buf, rec);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, rec, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return fail(ADMM_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
    *status_out = (h != 0 && (int)(h >> 56) - 1 == DBG_SELFTEST) ? ADMM_EBOUNDS : ADMM_OK;
    *index_out = (long long)(h & 0x00FFFFFFFFFFFFFFull);
    return ADMM_OK;
#else
    *status_out = ADMM_OK;
    *index_out = -1;
    return fail(ADMM_EUNSUPPORTED, "built without bounds checks (build with debug_bounds for libadmm_debug.so)");
#endif
}

admm_status admm_selftest_barrier_timeout(long long spin_ns, int grid, int *status_out)
{
    g_err.clear();
    if (!status_out || grid < 1 || grid > 64 || spin_ns <= 0 || spin_ns > 5000000000LL)
        return fail(ADMM_EINVAL, "bad selftest arguments");
    unsigned *bar = nullptr;
    int *status = nullptr;
    CUDA_TRY(cudaMalloc(&bar, sizeof(unsigned)));
    cudaError_t e = cudaMalloc(&status, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(bar);
        return fail(ADMM_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    cudaMemset(bar, 0, sizeof(unsigned));
    cudaMemset(status, 0, sizeof(int));
    void *args[] = {(void *)&bar, (void *)&status, (void *)&spin_ns, nullptr};
    unsigned extra = 1;
    args[3] = (void *)&extra;
    e = cudaLaunchCooperativeKernel((void *)selftest_barrier_kernel, dim3(grid), dim3(32), args, 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int sv = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&sv, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(bar);
    cudaFree(status);
    if (e != cudaSuccess) return fail(ADMM_ECUDA, "selftest: %s", cudaGetErrorString(e));
    *status_out = sv;
    return ADMM_OK;
}

} // extern "C"

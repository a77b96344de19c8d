// Host side of the batched solver API (admm_batch_* in include/admm.h):
// packing of many instances into one store, the launch configuration and
// its autotuner, CUDA-graph capture of the launch, and per-instance results.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "store.h"
#include "trace.h"

using namespace admm_impl;

namespace {

admm_status bfail(admm_status s, const std::string &msg)
{
    set_last_error(msg.c_str());
    return s;
}

#define BTRY(call)                                                                                        \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return bfail(e_ == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA,                       \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                             \
    } while (0)

// Host copy of a problem whose arrays may live on the device.
struct HostProblem {
    std::vector<double> a[10];
    admm_problem P{};
};
cudaError_t to_host(const admm_problem &in, HostProblem &out)
{
    out.P = in;
    if (!in.on_device) return cudaSuccess;
    // coefficient arrays: [m][q][n], or [m][n] when shared by the scenarios
    const size_t ne = (size_t)in.m * (in.coef_shared ? 1 : in.q) * in.n, nb = (size_t)in.m * in.n,
                 nc = (size_t)in.q * in.n;
    const double *src[10] = {in.f2, in.f1, in.f0, in.g2, in.g1, in.g0, in.x_lo, in.x_hi, in.y, in.c};
    const size_t cnt[10] = {ne, ne, ne, ne, ne, ne, nb, nb, nc, (size_t)in.m};
    const double **dst[10] = {&out.P.f2, &out.P.f1, &out.P.f0, &out.P.g2, &out.P.g1, &out.P.g0,
                              &out.P.x_lo, &out.P.x_hi, &out.P.y, &out.P.c};
    for (int t = 0; t < 10; ++t) {
        out.a[t].resize(cnt[t]);
        cudaError_t e = cudaMemcpy(out.a[t].data(), src[t], cnt[t] * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        *dst[t] = out.a[t].data();
    }
    out.P.on_device = 0;
    return cudaSuccess;
}

} // namespace

namespace admm_impl {

// Settings a batch or server accepts (the rules of admm_create, ADMM_MIXED only).
bool batch_params_ok(const admm_params *p, std::string &why)
{
    if (!p) {
        why = "params is NULL";
        return false;
    }
    for (int t = 0; t < 4; ++t)
        if (!(p->rho[t] > 0.0) || !std::isfinite(p->rho[t])) {
            why = "rho must be finite and > 0";
            return false;
        }
    if (p->max_iter < 1 || p->check_every < 1) {
        why = "max_iter and check_every must be >= 1";
        return false;
    }
    if (p->precision != ADMM_MIXED) {
        why = "the batched solver runs ADMM_MIXED only";
        return false;
    }
    if ((p->xmin_mode != ADMM_XMIN_EXACT && p->xmin_mode != ADMM_XMIN_PAPER) ||
        (p->sweep != ADMM_GAUSS_SEIDEL && p->sweep != ADMM_JACOBI) || (p->adapt_rho && !(p->tau > 1.0)) ||
        p->adapt_start < 0) {
        why = "bad xmin_mode, sweep, tau or adapt_start";
        return false;
    }
    if (!(p->r_tol >= 0.0) || !(p->s_tol >= 0.0) || p->reserved[0] || p->reserved[1]) {
        why = "r_tol, s_tol must be >= 0 and reserved fields 0";
        return false;
    }
    return true;
}

} // namespace admm_impl

struct admm_batch {
    int count = 0, dev = 0, nsm = 0, max_m = 0, max_q = 0;
    admm_params prm{};
    admm_batch_config cfg{8, 0, 0, 1, 0, 131072};
    Store store;
    std::vector<BatchInst> inst;
    BatchInst *d_inst = nullptr;
    int *d_order = nullptr; // orderL then orderS
    int *d_q = nullptr;     // three queue heads
    double *d_out = nullptr, *h_out = nullptr;
    double *d_tmp = nullptr;
    int nX = 0, nL = 0, nS = 0, cluster = 1;
    size_t slice = 0, smem = 0;
    int stage_off = 0;       // byte offset of the coefficient stages in a CTA's shared memory
    int grid = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int iter_budget = 0;
};

namespace {

void batch_free(admm_batch *b)
{
    b->store.free_all();
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_q) cudaFree(b->d_q);
    if (b->d_out) cudaFree(b->d_out);
    if (b->d_tmp) cudaFree(b->d_tmp);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
}

// Queues for the current configuration: CTA teams for instances above the
// small threshold, warp teams for the rest; each sorted by decreasing work.
admm_status build_queues(admm_batch *b)
{
    std::vector<int> X, L, S;
    const bool clusters = b->cfg.cluster_size > 1;
    for (int t = 0; t < b->count; ++t) {
        const int64_t el = (int64_t)b->inst[t].m * b->inst[t].q * b->inst[t].n;
        if (clusters && el > b->cfg.cluster_min_elements) X.push_back(t);
        else if (el > b->cfg.small_max_elements) L.push_back(t);
        else S.push_back(t);
    }
    auto work = [&](int t) { return (int64_t)b->inst[t].m * b->inst[t].q * b->inst[t].ld; };
    auto by_work = [&](int u, int v) { return work(u) != work(v) ? work(u) > work(v) : u < v; };
    std::sort(X.begin(), X.end(), by_work);
    std::sort(L.begin(), L.end(), by_work);
    std::sort(S.begin(), S.end(), by_work);
    b->nX = (int)X.size();
    b->nL = (int)L.size();
    b->nS = (int)S.size();
    std::vector<int> all(X);
    all.insert(all.end(), L.begin(), L.end());
    all.insert(all.end(), S.begin(), S.end());
    BTRY(cudaMemcpy(b->d_order, all.data(), sizeof(int) * std::max<size_t>(all.size(), 1), cudaMemcpyHostToDevice));
    // launch shape: as many co-resident CTAs (clusters) as fit
    const int mb = batch_mbound(b->max_m);
    // per-warp slices only when some instance runs on a one-warp team: the
    // shared memory left unclaimed serves as L1
    const BatchSmem bs = batch_cta_smem(b->max_m, b->max_q, b->cfg.warps_per_cta, clusters ? b->cfg.cluster_size : 1,
                                        b->nS > 0, b->slice);
    b->smem = bs.bytes;
    b->stage_off = bs.stage_off;
    const int per_sm = batch_blocks_per_sm(b->cfg.warps_per_cta, mb, b->smem, true);
    if (per_sm < 1) return bfail(ADMM_EUNSUPPORTED, "batched kernel cannot be resident with this configuration");
    const int use = b->cfg.ctas_per_sm > 0 ? std::min(b->cfg.ctas_per_sm, per_sm) : per_sm;
    b->cluster = clusters ? b->cfg.cluster_size : 1;
    if (b->cluster > 1) {
        const int nc = batch_max_clusters(b->cfg.warps_per_cta, mb, b->cluster, b->smem, true);
        if (nc < 1) return bfail(ADMM_EUNSUPPORTED, "clusters of this size cannot be resident");
        b->grid = std::min(nc, b->nsm * use / b->cluster) * b->cluster;
        if (b->grid < b->cluster) b->grid = b->cluster;
    } else {
        b->grid = b->nsm * use;
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return ADMM_OK;
}

BatchArgs make_args(const admm_batch *b)
{
    BatchArgs a{};
    a.inst = b->d_inst;
    a.orderX = b->d_order;
    a.orderL = b->d_order + b->nX;
    a.orderS = b->d_order + b->nX + b->nL;
    a.nX = b->nX;
    a.nL = b->nL;
    a.nS = b->nS;
    a.qX = b->d_q;
    a.qL = b->d_q + 1;
    a.qS = b->d_q + 2;
    a.dbg = (unsigned long long *)(b->d_q + 4);
    b->store.fill_args(a);
    a.f0 = b->store.f0;
    a.out = b->d_out;
    a.slice_doubles = (int)b->slice;
    a.stage_off = b->stage_off;
    a.iter_budget = b->iter_budget;
    a.r_tol = stop_r_tol(b->prm.precision, b->prm.r_tol);
    a.s_tol = stop_s_tol(b->prm.precision, b->prm.s_tol);
    a.adapt_target = b->prm.r_tol / b->prm.s_tol;
    a.adapt_start = b->prm.adapt_start;
    a.tau = b->prm.tau;
    a.max_iter = b->prm.max_iter;
    a.check_every = b->prm.check_every;
    a.xmin_mode = b->prm.xmin_mode;
    a.sweep = b->prm.sweep;
    a.adapt = b->prm.adapt_rho;
    return a;
}

// Captures {reset queue heads, batched kernel} into a CUDA graph once per
// configuration; later solves replay it.
admm_status ensure_graph(admm_batch *b)
{
    if (b->exec) return ADMM_OK;
    const BatchArgs a = make_args(b);
    cudaGraph_t g = nullptr;
    BTRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->d_q, 0, 4 * sizeof(int) + sizeof(unsigned long long), b->cap);
    if (e == cudaSuccess)
        e = launch_batch(b->cfg.warps_per_cta, batch_mbound(b->max_m), b->grid, b->cluster, a, b->smem, true, b->cap);
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(ADMM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(ADMM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return ADMM_OK;
}

admm_status reset_all(admm_batch *b)
{
    // zero start for every instance: x = clamp(0), s = mu = 0, scalar state
    // zero with rho, cold = 1; cleared records.
    std::vector<double> sc(b->store.cap_s, 0.0);
    for (int t = 0; t < b->count; ++t) {
        const BatchInst &I = b->inst[t];
        const int mq = I.m * I.q;
        double *p = sc.data() + I.off_scal;
        for (int u = 0; u < 4; ++u) p[5 * mq + I.m + u] = b->prm.rho[u];
        if (b->prm.rho2_over_n) p[5 * mq + I.m + 1] = b->prm.rho[1] / (double)I.n;
        p[5 * mq + I.m + 4] = 1.0;
        p[5 * mq + I.m + 5] = 1.0;
    }
    BTRY(cudaMemcpy(b->store.scal, sc.data(), sizeof(double) * sc.size(), cudaMemcpyHostToDevice));
    float *zc[4] = {b->store.s, b->store.s_lo, b->store.mu, b->store.mu_lo};
    for (float *a : zc) BTRY(cudaMemset(a, 0, sizeof(float) * b->store.cap_c));
    BTRY(cudaMemset(b->d_out, 0, sizeof(double) * kInfo * b->count));
    return ADMM_OK;
}

__global__ void batch_reset_x(const BatchInst *inst, int count, const float *lo, const float *hi, float *x)
{
    for (int id = blockIdx.x; id < count; id += gridDim.x) {
        const BatchInst I = inst[id];
        const int64_t tot = (int64_t)I.m * I.q * I.ld;
        for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
            const int k = (int)(t % I.ld);
            const int i = (int)(t / ((int64_t)I.q * I.ld));
            const float l = lo[I.off_b + (int64_t)i * I.ld + k], h = hi[I.off_b + (int64_t)i * I.ld + k];
            x[I.off_e + t] = 0.0f < l ? l : (0.0f > h ? h : 0.0f);
        }
    }
}

} // namespace

extern "C" {

admm_status admm_batch_create(const admm_problem *probs, int32_t count, const admm_params *prm, admm_batch **out)
{
    TraceRange trace_("admm_batch_create");
    clear_last_error();
    if (!out) return bfail(ADMM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!probs || count < 1) return bfail(ADMM_EINVAL, "need at least one problem");
    std::string why;
    if (!batch_params_ok(prm, why)) return bfail(prm && prm->precision != ADMM_MIXED ? ADMM_EUNSUPPORTED : ADMM_EINVAL, why);
    admm_batch *b = new admm_batch();
    b->count = count;
    b->prm = *prm;
    auto bail = [&](admm_status s) {
        batch_free(b);
        delete b;
        return s;
    };
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev);
    if (e != cudaSuccess) return bail(bfail(ADMM_ECUDA, cudaGetErrorString(e)));
    InstSizes tot{0, 0, 0, 0, 0, 0};
    size_t max_floats = 0, max_dense = 0;
    for (int t = 0; t < count; ++t) {
        const admm_problem &P = probs[t];
        if (P.n < 1 || P.m < 1 || P.q < 1) return bail(bfail(ADMM_EINVAL, "n, m, q must be >= 1"));
        if (P.m > ADMM_MAX_M || (int64_t)P.m * P.q > ADMM_BATCH_MAX_PAIRS)
            return bail(bfail(ADMM_EUNSUPPORTED, "instance " + std::to_string(t) + " exceeds m <= 8, m*q <= 256"));
        const InstSizes z = inst_sizes(P.n, P.m, P.q);
        tot.e += (z.e + 3) / 4 * 4;
        tot.b += (z.b + 3) / 4 * 4;
        tot.c += (z.c + 3) / 4 * 4;
        tot.p += z.p;
        tot.s += z.s;
        tot.m += z.m;
        max_floats = std::max(max_floats, (size_t)(7 * z.e + 2 * z.b + z.c));
        max_dense = std::max(max_dense, (size_t)P.m * P.q * P.n);
        b->max_m = std::max(b->max_m, P.m);
        b->max_q = std::max(b->max_q, P.q);
    }
    if (tot.e > kBatchArrayMax || tot.b > kBatchArrayMax || tot.c > kBatchArrayMax)
        return bail(bfail(ADMM_EUNSUPPORTED, "batch exceeds 2^32 - 1 elements per array: split it"));
    e = b->store.allocate(tot.e, tot.b, tot.c, tot.p, tot.s, tot.m);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_inst, sizeof(BatchInst) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_q, 4 * sizeof(int) + sizeof(unsigned long long)); // + bounds record
    if (e == cudaSuccess) e = cudaMalloc(&b->d_out, sizeof(double) * kInfo * count);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tmp, sizeof(double) * std::max<size_t>(max_dense, 1));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_out, sizeof(double) * kInfo * count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return bail(bfail(e == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA, cudaGetErrorString(e)));
    // The store's allocator places the instances in order; then worker threads validate, stage in
    // FP32 and upload them, each with its own stream and pinned staging buffer (the instances'
    // ranges are disjoint). The first error stops the workers and is the one reported.
    b->inst.resize(count);
    for (int t = 0; t < count; ++t)
        if (!b->store.place(probs[t].n, probs[t].m, probs[t].q, b->inst[t])) return bail(bfail(ADMM_ENOMEM, "store is full"));
    const int hw = (int)std::thread::hardware_concurrency();
    const int nthr = std::max(1, std::min(std::min(16, hw > 0 ? hw : 1), count));
    std::atomic<int> next{0};
    std::atomic<bool> failed{false};
    std::mutex emu;
    admm_status fst = ADMM_OK;
    std::string fmsg;
    auto fail_once = [&](admm_status s, const std::string &msg) {
        std::lock_guard<std::mutex> lk(emu);
        if (!failed.exchange(true)) {
            fst = s;
            fmsg = msg;
        }
    };
    auto worker = [&]() {
        cudaStream_t st = nullptr;
        float *pinned = nullptr;
        cudaError_t we = cudaSetDevice(b->dev);
        if (we == cudaSuccess) we = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (we == cudaSuccess) we = cudaMallocHost(&pinned, sizeof(float) * std::max<size_t>(max_floats, 4));
        if (we != cudaSuccess)
            fail_once(we == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA,
                      std::string("staging: ") + cudaGetErrorString(we));
        Staged S;
        HostProblem H;
        std::string wwhy;
        while (!failed.load()) {
            const int t = next.fetch_add(1);
            if (t >= count) break;
            we = to_host(probs[t], H);
            if (we != cudaSuccess) {
                fail_once(ADMM_ECUDA, cudaGetErrorString(we));
                break;
            }
            if (!stage_instance(H.P, S, wwhy)) {
                fail_once(ADMM_EINVAL, "instance " + std::to_string(t) + ": " + wwhy);
                break;
            }
            b->inst[t].cs = S.cs;
            we = b->store.upload(b->inst[t], S, b->prm, pinned, max_floats, st);
            if (we != cudaSuccess) {
                fail_once(ADMM_ECUDA, cudaGetErrorString(we));
                break;
            }
        }
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        if (pinned) cudaFreeHost(pinned);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nthr; ++w) pool.emplace_back(worker);
    for (std::thread &th : pool) th.join();
    if (failed.load()) return bail(bfail(fst, fmsg));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_out, 0, sizeof(double) * kInfo * count);
    if (e != cudaSuccess) return bail(bfail(ADMM_ECUDA, cudaGetErrorString(e)));
    b->slice = batch_slice_doubles(b->max_m, b->max_q);
    admm_status s = build_queues(b);
    if (s != ADMM_OK) return bail(s);
    *out = b;
    return ADMM_OK;
}

admm_status admm_batch_set_config(admm_batch *b, const admm_batch_config *cfg)
{
    clear_last_error();
    if (!b || !cfg) return bfail(ADMM_EINVAL, "NULL argument");
    if (cfg->warps_per_cta != 4 && cfg->warps_per_cta != 8 && cfg->warps_per_cta != 16)
        return bfail(ADMM_EINVAL, "warps_per_cta must be 4, 8 or 16");
    if (cfg->ctas_per_sm < 0 || cfg->small_max_elements < 0 || cfg->cluster_min_elements < 0)
        return bfail(ADMM_EINVAL, "negative setting");
    if (cfg->cluster_size != 1 && cfg->cluster_size != 2 && cfg->cluster_size != 4 && cfg->cluster_size != 8)
        return bfail(ADMM_EINVAL, "cluster_size must be 1, 2, 4 or 8");
    if (cfg->reserved) return bfail(ADMM_EINVAL, "reserved must be 0");
    b->cfg = *cfg;
    return build_queues(b);
}

admm_status admm_batch_get_config(admm_batch *b, admm_batch_config *cfg)
{
    if (!b || !cfg) return bfail(ADMM_EINVAL, "NULL argument");
    *cfg = b->cfg;
    cfg->ctas_per_sm = (b->grid + b->nsm - 1) / std::max(1, b->nsm);
    return ADMM_OK;
}

admm_status admm_batch_solve(admm_batch *b, void *stream)
{
    TraceRange trace_("admm_batch_solve");
    clear_last_error();
    if (!b) return bfail(ADMM_EINVAL, "batch is NULL");
    admm_status s = ensure_graph(b);
    if (s != ADMM_OK) return s;
    BTRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return ADMM_OK;
}

admm_status admm_batch_wait(admm_batch *b, void *stream, admm_result *results)
{
    clear_last_error();
    if (!b) return bfail(ADMM_EINVAL, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    BTRY(cudaMemcpyAsync(b->h_out, b->d_out, sizeof(double) * kInfo * b->count, cudaMemcpyDeviceToHost, st));
    unsigned long long rec = 0; // bounds record of checked builds
    BTRY(cudaMemcpyAsync(&rec, b->d_q + 4, sizeof rec, cudaMemcpyDeviceToHost, st));
    BTRY(cudaStreamSynchronize(st));
    if (rec != 0)
        return bfail(ADMM_EBOUNDS, "element access out of bounds: array " + std::to_string((int)(rec >> 56) - 1) +
                                       ", index " + std::to_string((long long)(rec & 0x00FFFFFFFFFFFFFFull)));
    admm_status worst = ADMM_OK;
    for (int t = 0; t < b->count; ++t) {
        const double *o = b->h_out + (size_t)t * kInfo;
        admm_status s = o[12] != 0.0 ? (admm_status)(int)o[12] : (o[1] != 0.0 ? ADMM_OK : ADMM_ENOTCONVERGED);
        if (s != ADMM_OK && worst == ADMM_OK) worst = s;
        if (!results) continue;
        admm_result &r = results[t];
        r.iters = (int32_t)o[0];
        r.converged = o[1] != 0.0;
        r.r = o[2];
        r.sigma = o[3];
        r.objective = o[11];
        r.status = s;
        if (r.x || r.x1) {
            admm_state st_out{};
            st_out.x = r.x;
            st_out.x1 = r.x1;
            st_out.on_device = r.on_device;
            BTRY(store_get_state(b->store, b->inst[t], &st_out, b->d_tmp, st));
        }
    }
    return worst;
}

admm_status admm_batch_get_info(admm_batch *b, int32_t idx, double *info, int32_t count)
{
    clear_last_error();
    if (!b || !info || idx < 0 || idx >= b->count || count < 1) return bfail(ADMM_EINVAL, "bad argument");
    for (int t = 0; t < count && t < kInfo; ++t) info[t] = b->h_out[(size_t)idx * kInfo + t];
    return ADMM_OK;
}

admm_status admm_batch_get_state(admm_batch *b, int32_t idx, admm_state *out)
{
    clear_last_error();
    if (!b || !out || idx < 0 || idx >= b->count) return bfail(ADMM_EINVAL, "bad argument");
    BTRY(store_get_state(b->store, b->inst[idx], out, b->d_tmp, b->cap));
    return ADMM_OK;
}

admm_status admm_batch_set_state(admm_batch *b, int32_t idx, const admm_state *in)
{
    clear_last_error();
    if (!b || !in || idx < 0 || idx >= b->count) return bfail(ADMM_EINVAL, "bad argument");
    if (!in->x || !in->s || !in->mu || !in->lam || !in->zeta || !in->h || !in->p || !in->nu || !in->x1)
        return bfail(ADMM_EINVAL, "state has a NULL array");
    BTRY(store_set_state(b->store, b->inst[idx], in, b->d_tmp, b->cap));
    BTRY(cudaMemset(b->d_out + (size_t)idx * kInfo, 0, sizeof(double) * kInfo));
    return ADMM_OK;
}

admm_status admm_batch_reset(admm_batch *b)
{
    clear_last_error();
    if (!b) return bfail(ADMM_EINVAL, "batch is NULL");
    batch_reset_x<<<std::min(b->count, b->nsm * 8), 256>>>(b->d_inst, b->count, b->store.lo, b->store.hi, b->store.x);
    BTRY(cudaGetLastError());
    admm_status s = reset_all(b);
    if (s != ADMM_OK) return s;
    BTRY(cudaDeviceSynchronize());
    return ADMM_OK;
}

admm_status admm_batch_autotune(admm_batch *b, int32_t trial_iters, admm_batch_config *chosen)
{
    TraceRange trace_("admm_batch_autotune");
    clear_last_error();
    if (!b || trial_iters < 0) return bfail(ADMM_EINVAL, "bad argument");
    const admm_batch_config keep = b->cfg;
    // trial_iters > 0: throughput over that many iterations; 0: whole solves,
    // whose time includes the tail of the slowest instances (where multi-CTA
    // cluster teams for the largest instances pay)
    const bool whole = trial_iters == 0;
    const std::vector<int64_t> thresholds = whole ? std::vector<int64_t>{0} : std::vector<int64_t>{0, 8192, 32768};
    const std::vector<int> warps = whole ? std::vector<int>{8, 16} : std::vector<int>{4, 8, 16};
    struct Clus {
        int32_t size;
        int64_t min_el;
    };
    const std::vector<Clus> clus = whole ? std::vector<Clus>{{1, 0}, {2, 100000}, {2, 150000}, {2, 250000}, {4, 250000}}
                                         : std::vector<Clus>{{1, 0}, {4, 131072}, {8, 131072}, {8, 32768}};
    cudaEvent_t e0, e1;
    BTRY(cudaEventCreate(&e0));
    BTRY(cudaEventCreate(&e1));
    float best = 1e30f;
    admm_batch_config best_cfg = keep;
    b->iter_budget = trial_iters;
    for (int w : warps)
        for (int64_t th : thresholds)
            for (const Clus &cc : clus) {
                if (cc.size > 1 && cc.min_el < th) continue;
                admm_batch_config c{w, 0, th, cc.size, 0, cc.min_el};
                b->cfg = c;
                if (build_queues(b) != ADMM_OK) continue;
                if (admm_batch_reset(b) != ADMM_OK) break;
                const BatchArgs a = make_args(b);
                cudaMemset(b->d_q, 0, 3 * sizeof(int));
                cudaEventRecord(e0, b->cap);
                cudaError_t e = launch_batch(w, batch_mbound(b->max_m), b->grid, b->cluster, a, b->smem, true, b->cap);
                cudaEventRecord(e1, b->cap);
                if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_cfg = c;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->iter_budget = 0;
    b->cfg = best_cfg;
    admm_status s = build_queues(b);
    if (s == ADMM_OK) s = admm_batch_reset(b);
    if (s == ADMM_OK && chosen) admm_batch_get_config(b, chosen);
    return s;
}

admm_status admm_batch_destroy(admm_batch *b)
{
    if (!b) return ADMM_OK;
    batch_free(b);
    delete b;
    return ADMM_OK;
}

} // extern "C"

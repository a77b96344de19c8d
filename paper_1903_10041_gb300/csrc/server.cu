// Serving: continuous batching of MPC re-solves (admm_server_* in admm.h).
//
// Requests (a problem, optionally tied to a session = one controller) are
// validated and packed to FP32 on the submitting thread, then queued.  A
// worker thread runs ticks: it admits queued requests in arrival order
// while the device store has room and a slot is free (memory-based
// admission; idle sessions are evicted least-recently-used first when the
// store is full), replays a CUDA graph that runs the batched kernel on every
// active instance (the costliest one for `tick_iters` iterations, the others
// for as many as fit in the same time; in round-robin slices when instances
// outnumber the CTA teams), and retires the instances that finished
// (converged or out of iterations), gathering their results to the host
// with one kernel and one copy.  Requests that arrive while others are on
// the GPU join at the next tick.  A session keeps its instance's state resident on the device
// after a solve; the next request of that session is warm-started from it,
// moved one step forward on the device (the receding horizon of Sec. II and
// Alg. 2).  An instance's arithmetic depends only on its own shape and team
// kind, so its result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "store.h"
#include "trace.h"

using namespace admm_impl;

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0, session = -1;
    Staged staged;               // full problem (is_step == false)
    bool is_step = false;        // receding-horizon step of a resident session
    int step_m = 0, step_q = 0;
    std::vector<float> payload;  // step data: f2 f1 f0 g2 g1 g0 [m][q], lo hi [m], y [q]
    double t_submit = 0, t_admit = 0, t_finish = 0;
    int slot = -1;
    bool warm = false, done = false, cancel = false;
    admm_status status = ADMM_OK;
    double info[kInfo] = {};
    std::vector<double> x, x1;
};

struct Session {
    BatchInst inst{};
    bool resident = false;
    bool busy = false;
    double last_used = 0;
};

} // namespace

struct admm_server {
    admm_params prm{};
    admm_server_config cfg{};
    int dev = 0, nsm = 0, grid = 0, mbound = 8, cluster = 1;
    size_t slice = 0, smem = 0;
    int stage_off = 0;       // byte offset of the coefficient stages in a CTA's shared memory
    Store store;
    cudaStream_t st = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchInst *d_inst = nullptr, *h_inst = nullptr;
    int *d_order = nullptr, *h_order = nullptr; // [0, max) cluster, [max, 2 max) CTA, [2 max, 3 max) warp teams
    int *d_counts = nullptr, *h_counts = nullptr, *d_q = nullptr;
    int *d_shift = nullptr, *h_shift = nullptr;
    int *d_stepids = nullptr, *h_stepids = nullptr;
    float *d_payload = nullptr, *h_payload = nullptr;
    int payload_stride = 0;
    double *d_out = nullptr, *h_out = nullptr, *d_tmp = nullptr;
    size_t tmp_n = 0;
    int *d_gids = nullptr, *h_gids = nullptr;       // finished instances of a tick
    int *d_lock = nullptr;                          // per slot: a team runs it (round-robin ticks)
    int64_t *d_goff = nullptr, *h_goff = nullptr;   // their offsets in the gathered results
    double *h_gather = nullptr;                     // gathered x and x_1 (pinned)
    size_t gather_n = 0;
    float *pinned = nullptr;
    size_t pinned_n = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::map<int64_t, std::shared_ptr<Request>> reqs;
    std::vector<std::shared_ptr<Request>> active; // by slot
    std::vector<int> free_slots;
    std::map<int64_t, Session> sessions;
    int64_t next_ticket = 1;
    bool stop = false;
    double stats[8] = {}; // ticks, admitted, finished, GPU seconds in ticks, GPU seconds in step shifts,
                          // sum over ticks of the instances in the tick
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::string worker_error;
    std::thread worker;
};

namespace {

admm_status sfail(admm_status s, const std::string &msg)
{
    set_last_error(msg.c_str());
    return s;
}

cudaError_t ensure_tmp(admm_server *S, size_t n)
{
    if (S->tmp_n >= n) return cudaSuccess;
    if (S->d_tmp) cudaFree(S->d_tmp);
    S->d_tmp = nullptr;
    S->tmp_n = 0;
    cudaError_t e = cudaMalloc(&S->d_tmp, n * sizeof(double));
    if (e == cudaSuccess) S->tmp_n = n;
    return e;
}

cudaError_t ensure_gather(admm_server *S, size_t n)
{
    cudaError_t e = ensure_tmp(S, n);
    if (e != cudaSuccess || S->gather_n >= n) return e;
    if (S->h_gather) cudaFreeHost(S->h_gather);
    S->h_gather = nullptr;
    S->gather_n = 0;
    e = cudaMallocHost(&S->h_gather, n * sizeof(double));
    if (e == cudaSuccess) S->gather_n = n;
    return e;
}

cudaError_t ensure_pinned(admm_server *S, size_t n)
{
    if (S->pinned_n >= n) return cudaSuccess;
    if (S->pinned) cudaFreeHost(S->pinned);
    S->pinned = nullptr;
    S->pinned_n = 0;
    cudaError_t e = cudaMallocHost(&S->pinned, n * sizeof(float));
    if (e == cudaSuccess) S->pinned_n = n;
    return e;
}

// Reserves store room for a request, evicting idle resident sessions
// (least recently used first) when needed.  Caller holds no lock; only the
// worker thread touches the store and sessions' allocations.
bool place_with_eviction(admm_server *S, const Staged &st, BatchInst &I, int64_t keep_session)
{
    for (;;) {
        if (S->store.place(st.n, st.m, st.q, I)) return true;
        int64_t victim = -1;
        double oldest = 1e300;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto &kv : S->sessions)
                if (kv.first != keep_session && kv.second.resident && !kv.second.busy && kv.second.last_used < oldest) {
                    oldest = kv.second.last_used;
                    victim = kv.first;
                }
            if (victim < 0) return false;
            S->store.release(S->sessions[victim].inst);
            S->sessions[victim].resident = false;
        }
    }
}

void worker_loop(admm_server *S)
{
    cudaSetDevice(S->dev);
    const int maxa = S->cfg.max_active;
    std::vector<int> shift_ids;
    for (;;) {
        std::vector<std::shared_ptr<Request>> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                const bool any_active = std::any_of(S->active.begin(), S->active.end(), [](auto &p) { return (bool)p; });
                return S->stop || any_active || !S->pending.empty();
            });
            if (S->stop) return;
            // Admission in arrival order while slots are free.  A request of
            // a session with a solve in flight (or admitted earlier in this
            // pass) stays queued, keeping its session's order, without
            // blocking the requests of other sessions behind it.
            for (auto it = S->pending.begin(); it != S->pending.end() && !S->free_slots.empty();) {
                auto r = *it;
                if (r->session >= 0 && S->sessions[r->session].busy) {
                    ++it;
                    continue;
                }
                it = S->pending.erase(it);
                if (r->session >= 0) S->sessions[r->session].busy = true;
                admit.push_back(r);
                r->slot = S->free_slots.back();
                S->free_slots.pop_back();
            }
        }
        // place and upload the admitted requests (worker-only state)
        shift_ids.clear();
        bool inst_dirty = false, shift_timed = false;
        std::vector<std::shared_ptr<Request>> back_to_queue;
        std::vector<int> step_ids;
        for (auto &r : admit) {
            if (r->is_step) {
                BatchInst I{};
                bool ok = false;
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    Session &ss = S->sessions[r->session];
                    if (ss.resident && ss.inst.m == r->step_m && ss.inst.q == r->step_q) {
                        I = ss.inst;
                        ok = true;
                    }
                }
                if (!ok) { // the session has no resident instance of that shape
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->free_slots.push_back(r->slot);
                    r->slot = -1;
                    S->sessions[r->session].busy = false;
                    r->status = ADMM_EINVAL;
                    r->done = true;
                    r->t_finish = now_s();
                    S->cv_done.notify_all();
                    continue;
                }
                // staged in admission order; one copy for all of them below
                std::memcpy(S->h_payload + step_ids.size() * S->payload_stride, r->payload.data(),
                            sizeof(float) * r->payload.size());
                S->h_inst[r->slot] = I;
                inst_dirty = true;
                step_ids.push_back(r->slot);
                r->warm = true;
                r->t_admit = now_s();
                std::lock_guard<std::mutex> lk(S->mu);
                S->active[r->slot] = r;
                S->stats[1] += 1;
                continue;
            }
            const Staged &sg = r->staged;
            BatchInst I{};
            bool reuse = false;
            if (r->session >= 0) {
                std::lock_guard<std::mutex> lk(S->mu);
                Session &ss = S->sessions[r->session];
                if (ss.resident && ss.inst.n == sg.n && ss.inst.m == sg.m && ss.inst.q == sg.q &&
                    ss.inst.cs == sg.cs) {
                    I = ss.inst;
                    reuse = true;
                }
            }
            if (!reuse && !place_with_eviction(S, sg, I, r->session)) {
                back_to_queue.push_back(r); // store full: wait for a later tick
                continue;
            }
            I.cs = sg.cs;
            const InstSizes z = inst_sizes(sg.n, sg.m, sg.q);
            cudaError_t e = ensure_pinned(S, 7 * (size_t)z.e + 2 * (size_t)z.b + (size_t)z.c);
            if (e == cudaSuccess) {
                if (reuse) {
                    // new problem data, but keep x, s, mu and the scalar state
                    const Staged &keep = sg; // f, g, bounds, y and c are replaced; x, s, mu, scalars kept
                    float *dst_e[6] = {S->store.f2, S->store.f1, S->store.f0, S->store.g2, S->store.g1, S->store.g0};
                    e = cudaStreamSynchronize(S->st);
                    size_t at = 0;
                    for (int t = 0; t < 6 && e == cudaSuccess; ++t) {
                        std::memcpy(S->pinned + at, keep.e[t].data(), sizeof(float) * z.e);
                        e = cudaMemcpyAsync(dst_e[t] + I.off_e, S->pinned + at, sizeof(float) * z.e,
                                            cudaMemcpyHostToDevice, S->st);
                        at += z.e;
                    }
                    float *dst_b[2] = {S->store.lo, S->store.hi};
                    for (int t = 0; t < 2 && e == cudaSuccess; ++t) {
                        std::memcpy(S->pinned + at, keep.b[t].data(), sizeof(float) * z.b);
                        e = cudaMemcpyAsync(dst_b[t] + I.off_b, S->pinned + at, sizeof(float) * z.b,
                                            cudaMemcpyHostToDevice, S->st);
                        at += z.b;
                    }
                    if (e == cudaSuccess) {
                        std::memcpy(S->pinned + at, keep.y.data(), sizeof(float) * z.c);
                        e = cudaMemcpyAsync(S->store.y + I.off_c, S->pinned + at, sizeof(float) * z.c,
                                            cudaMemcpyHostToDevice, S->st);
                    }
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(S->store.sumg0 + I.off_pair, keep.sumg0.data(), sizeof(double) * z.p,
                                            cudaMemcpyHostToDevice, S->st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(S->store.c + I.off_src, keep.c.data(), sizeof(double) * z.m,
                                            cudaMemcpyHostToDevice, S->st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
                    r->warm = true;
                    shift_ids.push_back(r->slot);
                } else {
                    e = S->store.upload(I, sg, S->prm, S->pinned, S->pinned_n, S->st);
                }
            }
            if (e != cudaSuccess) {
                if (!reuse) S->store.release(I);
                std::lock_guard<std::mutex> lk(S->mu);
                S->free_slots.push_back(r->slot);
                r->slot = -1;
                if (r->session >= 0) S->sessions[r->session].busy = false;
                S->worker_error = cudaGetErrorString(e);
                r->status = ADMM_ECUDA;
                r->done = true;
                r->t_finish = now_s();
                S->cv_done.notify_all();
                continue;
            }
            S->h_inst[r->slot] = I;
            inst_dirty = true;
            cudaMemsetAsync(S->d_out + (size_t)r->slot * kInfo, 0, sizeof(double) * kInfo, S->st);
            if (r->session >= 0) {
                std::lock_guard<std::mutex> lk(S->mu);
                Session &ss = S->sessions[r->session];
                ss.inst = I;
                ss.resident = true;
            }
            r->t_admit = now_s();
            std::lock_guard<std::mutex> lk(S->mu);
            S->active[r->slot] = r;
            S->stats[1] += 1;
        }
        if (!back_to_queue.empty()) {
            std::lock_guard<std::mutex> lk(S->mu);
            const bool any_active = std::any_of(S->active.begin(), S->active.end(), [](auto &p) { return (bool)p; });
            for (auto it = back_to_queue.rbegin(); it != back_to_queue.rend(); ++it) {
                S->free_slots.push_back((*it)->slot);
                (*it)->slot = -1;
                if ((*it)->session >= 0) S->sessions[(*it)->session].busy = false;
                if (any_active) {
                    S->pending.push_front(*it); // retried when running instances free the store
                } else {
                    // nothing runs and every idle session is evicted: it can never fit
                    (*it)->status = ADMM_ENOMEM;
                    (*it)->done = true;
                    (*it)->t_finish = now_s();
                }
            }
            S->cv_done.notify_all();
        }
        if (inst_dirty) // the whole instance table in one copy (a few hundred KB)
            cudaMemcpyAsync(S->d_inst, S->h_inst, sizeof(BatchInst) * maxa, cudaMemcpyHostToDevice, S->st);
        if (!step_ids.empty()) {
            std::copy(step_ids.begin(), step_ids.end(), S->h_stepids);
            cudaMemcpyAsync(S->d_stepids, S->h_stepids, sizeof(int) * step_ids.size(), cudaMemcpyHostToDevice, S->st);
            cudaMemcpyAsync(S->d_payload, S->h_payload, sizeof(float) * step_ids.size() * S->payload_stride,
                            cudaMemcpyHostToDevice, S->st);
            Store &T = S->store;
            cudaEventRecord(S->ev[2], S->st);
            launch_shift_step(S->d_inst, S->d_stepids, (int)step_ids.size(), S->d_payload, S->payload_stride, T.f2,
                              T.f1, T.f0, T.g2, T.g1, T.g0, T.lo, T.hi, T.y, T.x, T.s, T.s_lo, T.mu, T.mu_lo, T.sumg0,
                              T.scal, S->d_out, S->st);
            cudaEventRecord(S->ev[3], S->st);
            shift_timed = true;
        }
        if (!shift_ids.empty()) {
            std::copy(shift_ids.begin(), shift_ids.end(), S->h_shift);
            cudaMemcpyAsync(S->d_shift, S->h_shift, sizeof(int) * shift_ids.size(), cudaMemcpyHostToDevice, S->st);
            launch_shift_state(S->d_inst, S->d_shift, (int)shift_ids.size(), S->store.x, S->store.s, S->store.s_lo,
                               S->store.mu, S->store.mu_lo, S->store.scal, S->st);
        }
        TraceRange trace_("admm_server_tick");
        // cancelled requests leave at the tick boundary
        {
            std::lock_guard<std::mutex> lk(S->mu);
            bool any = false;
            for (int s = 0; s < maxa; ++s) {
                std::shared_ptr<Request> r = S->active[s];
                if (!r || !r->cancel) continue;
                if (r->session >= 0) {
                    Session &ss = S->sessions[r->session];
                    ss.busy = false;
                    ss.last_used = now_s();
                } else {
                    S->store.release(S->h_inst[s]);
                }
                S->active[s] = nullptr;
                S->free_slots.push_back(s);
                r->status = ADMM_ECANCELLED;
                r->t_finish = now_s();
                r->done = true;
                any = true;
            }
            if (any) S->cv_done.notify_all();
        }
        // queues of the active instances for this tick
        int nX = 0, nL = 0, nS = 0;
        std::vector<int> ids;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int s = 0; s < maxa; ++s)
                if (S->active[s]) ids.push_back(s);
        }
        auto work = [&](int s) { return (int64_t)S->h_inst[s].m * S->h_inst[s].q * S->h_inst[s].ld; };
        std::sort(ids.begin(), ids.end(), [&](int u, int v) { return work(u) != work(v) ? work(u) > work(v) : u < v; });
        for (int s : ids) {
            const int64_t el = (int64_t)S->h_inst[s].m * S->h_inst[s].q * S->h_inst[s].n;
            if (S->cluster > 1 && el > S->cfg.batch.cluster_min_elements) S->h_order[nX++] = s;
            else if (el > S->cfg.batch.small_max_elements) S->h_order[maxa + nL++] = s;
            else S->h_order[2 * maxa + nS++] = s;
        }
        if (ids.empty()) continue;
        S->h_counts[0] = nX;
        S->h_counts[1] = nL;
        S->h_counts[2] = nS;
        {   // time-balanced budgets: the largest per-thread cost of the tick sets its length
            float cmax = 0.0f;
            const int wc = S->cfg.batch.warps_per_cta * 32;
            for (int t = 0; t < nX + nL + nS; ++t) {
                const int s = t < nX ? S->h_order[t] : (t < nX + nL ? S->h_order[maxa + t - nX]
                                                                    : S->h_order[2 * maxa + t - nX - nL]);
                const int threads = t < nX ? S->cluster * wc : (t < nX + nL ? wc : 32);
                cmax = std::max(cmax, team_iter_cost(S->h_inst[s].n, S->h_inst[s].m, S->h_inst[s].q, threads));
            }
            // Round-robin slices when the CTA teams are outnumbered: the tick
            // keeps the length of ceil(A / teams) passes of the costliest
            // instance, cut into R slices per instance so no team idles in a
            // partial last round.  Cluster teams run their instances first
            // (one pass each, worth R slices), so the CTAs they hold are not
            // counted as CTA teams.
            int rounds = 1;
            float tw = (float)S->cfg.tick_iters * cmax;
            const int teams = std::max(1, S->grid - std::min(nX * S->cluster, S->grid / 2));
            if (nS == 0 && nL > teams) {
                rounds = 4;
                const int passes = (nL + teams - 1) / teams;
                tw = (float)((double)tw * passes * teams / ((double)nL * rounds));
            }
            std::memcpy(&S->h_counts[3], &tw, sizeof(float));
            S->h_counts[4] = rounds;
        }
        cudaMemcpyAsync(S->d_order, S->h_order, sizeof(int) * nX, cudaMemcpyHostToDevice, S->st);
        cudaMemcpyAsync(S->d_order + maxa, S->h_order + maxa, sizeof(int) * nL, cudaMemcpyHostToDevice, S->st);
        cudaMemcpyAsync(S->d_order + 2 * maxa, S->h_order + 2 * maxa, sizeof(int) * nS, cudaMemcpyHostToDevice, S->st);
        cudaMemcpyAsync(S->d_counts, S->h_counts, 5 * sizeof(int), cudaMemcpyHostToDevice, S->st);
        cudaEventRecord(S->ev[0], S->st);
        cudaError_t e = cudaGraphLaunch(S->exec, S->st);
        cudaEventRecord(S->ev[1], S->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->h_out, S->d_out, sizeof(double) * kInfo * maxa, cudaMemcpyDeviceToHost, S->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->st);
        float tick_ms = 0.0f;
        if (e == cudaSuccess && cudaEventElapsedTime(&tick_ms, S->ev[0], S->ev[1]) == cudaSuccess)
            S->stats[3] += 1e-3 * tick_ms;
        if (e == cudaSuccess && shift_timed && cudaEventElapsedTime(&tick_ms, S->ev[2], S->ev[3]) == cudaSuccess)
            S->stats[4] += 1e-3 * tick_ms;
        S->stats[0] += 1;
        S->stats[5] += (double)ids.size();
        // retire finished instances: their x and x_1 come back in one gather
        // kernel and one copy
        std::vector<int> fin;
        for (int s : ids)
            if (e != cudaSuccess || S->h_out[(size_t)s * kInfo + 14] != 0.0) fin.push_back(s);
        cudaError_t eg = cudaSuccess;
        if (e == cudaSuccess && !fin.empty()) {
            int64_t tot = 0;
            for (size_t t = 0; t < fin.size(); ++t) {
                const BatchInst &I = S->h_inst[fin[t]];
                S->h_gids[t] = fin[t];
                S->h_goff[t] = tot;
                tot += (int64_t)I.m * I.q * I.n + I.m;
            }
            eg = ensure_gather(S, (size_t)tot);
            if (eg == cudaSuccess)
                eg = cudaMemcpyAsync(S->d_gids, S->h_gids, sizeof(int) * fin.size(), cudaMemcpyHostToDevice, S->st);
            if (eg == cudaSuccess)
                eg = cudaMemcpyAsync(S->d_goff, S->h_goff, sizeof(int64_t) * fin.size(), cudaMemcpyHostToDevice,
                                     S->st);
            if (eg == cudaSuccess) {
                launch_gather_x(S->d_inst, S->d_gids, S->d_goff, (int)fin.size(), S->store.x, S->store.scal, S->d_tmp,
                                S->st);
                eg = cudaMemcpyAsync(S->h_gather, S->d_tmp, sizeof(double) * tot, cudaMemcpyDeviceToHost, S->st);
            }
            if (eg == cudaSuccess) eg = cudaStreamSynchronize(S->st);
        }
        for (size_t t = 0; t < fin.size(); ++t) {
            const int s = fin[t];
            const double *o = S->h_out + (size_t)s * kInfo;
            std::shared_ptr<Request> r;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                r = S->active[s];
            }
            const BatchInst I = S->h_inst[s];
            if (e == cudaSuccess) {
                std::memcpy(r->info, o, sizeof(double) * kInfo);
                const size_t nx = (size_t)I.m * I.q * I.n;
                r->x.resize(nx);
                r->x1.resize(I.m);
                if (eg == cudaSuccess) {
                    std::memcpy(r->x.data(), S->h_gather + S->h_goff[t], sizeof(double) * nx);
                    std::memcpy(r->x1.data(), S->h_gather + S->h_goff[t] + nx, sizeof(double) * I.m);
                }
                r->status = eg != cudaSuccess ? ADMM_ECUDA
                                              : (o[12] != 0.0 ? (admm_status)(int)o[12]
                                                              : (o[1] != 0.0 ? ADMM_OK : ADMM_ENOTCONVERGED));
            } else {
                r->status = ADMM_ECUDA;
                S->worker_error = cudaGetErrorString(e);
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (r->session >= 0) {
                Session &ss = S->sessions[r->session];
                ss.busy = false;
                ss.last_used = now_s();
            } else {
                S->store.release(I);
            }
            S->active[s] = nullptr;
            S->free_slots.push_back(s);
            r->t_finish = now_s();
            r->done = true;
            S->stats[2] += 1;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->cv_done.notify_all();
        }
    }
}

} // namespace

extern "C" {

void admm_server_default_config(admm_server_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->store_elements = 1LL << 27;
    c->max_active = 4096;
    c->tick_iters = 10;
    c->max_m = 4;
    c->max_q = 20;
    c->batch.warps_per_cta = 8;
    c->batch.ctas_per_sm = 0;
    c->batch.small_max_elements = 0;
    c->batch.cluster_size = 1;
    c->batch.cluster_min_elements = 131072;
}

admm_status admm_server_create(const admm_params *prm, const admm_server_config *cfg, admm_server **out)
{
    clear_last_error();
    if (!out || !prm || !cfg) return sfail(ADMM_EINVAL, "NULL argument");
    *out = nullptr;
    if (prm->precision != ADMM_MIXED) return sfail(ADMM_EUNSUPPORTED, "the server runs ADMM_MIXED only");
    if (cfg->max_active < 1 || cfg->tick_iters < 1 || cfg->store_elements < 1024 || cfg->max_m < 1 ||
        cfg->max_m > ADMM_MAX_M || cfg->max_q < 1 || (int64_t)cfg->max_m * cfg->max_q > ADMM_BATCH_MAX_PAIRS)
        return sfail(ADMM_EINVAL, "bad server configuration");
    if (cfg->store_elements > kBatchArrayMax)
        return sfail(ADMM_EUNSUPPORTED, "store_elements exceeds 2^32 - 1 (the kernel's 32-bit array offsets)");
    if (cfg->batch.warps_per_cta != 4 && cfg->batch.warps_per_cta != 8 && cfg->batch.warps_per_cta != 16)
        return sfail(ADMM_EINVAL, "warps_per_cta must be 4, 8 or 16");
    if (cfg->batch.cluster_size != 1 && cfg->batch.cluster_size != 2 && cfg->batch.cluster_size != 4 &&
        cfg->batch.cluster_size != 8)
        return sfail(ADMM_EINVAL, "cluster_size must be 1, 2, 4 or 8");
    if (cfg->batch.ctas_per_sm < 0 || cfg->batch.small_max_elements < 0 || cfg->batch.cluster_min_elements < 0)
        return sfail(ADMM_EINVAL, "negative setting");
    if (cfg->batch.reserved) return sfail(ADMM_EINVAL, "reserved must be 0");
    std::string why;
    if (!batch_params_ok(prm, why)) return sfail(ADMM_EINVAL, why); // the rules of admm_batch_create
    admm_server *S = new admm_server();
    S->prm = *prm;
    S->cfg = *cfg;
    const int maxa = cfg->max_active;
    auto bail = [&](admm_status s, const std::string &m) {
        S->store.free_all();
        void *d[] = {S->d_inst,  S->d_order, S->d_counts,  S->d_q,    S->d_shift, S->d_out,
                     S->d_tmp,   S->d_stepids, S->d_payload, S->d_gids, S->d_goff, S->d_lock};
        for (void *p : d)
            if (p) cudaFree(p);
        void *h[] = {S->h_inst,  S->h_order,   S->h_counts, S->h_shift, S->h_out,
                     S->pinned,  S->h_stepids, S->h_payload, S->h_gids, S->h_goff, S->h_gather};
        for (void *p : h)
            if (p) cudaFreeHost(p);
        if (S->st) cudaStreamDestroy(S->st);
        for (cudaEvent_t ev : S->ev)
            if (ev) cudaEventDestroy(ev);
        delete S;
        return sfail(s, m);
    };
    cudaError_t e = cudaGetDevice(&S->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, S->dev);
    const int64_t E = cfg->store_elements;
    if (e == cudaSuccess)
        e = S->store.allocate(E, E, E, (int64_t)maxa * cfg->max_m * cfg->max_q,
                              (int64_t)maxa * scal_size(cfg->max_m, cfg->max_q), (int64_t)maxa * cfg->max_m);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_inst, sizeof(BatchInst) * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_order, sizeof(int) * 3 * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_counts, sizeof(int) * 5); // nX, nL, nS, tick work (float), rounds
    if (e == cudaSuccess) e = cudaMalloc(&S->d_q, sizeof(int) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_shift, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_gids, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_goff, sizeof(int64_t) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_gids, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_goff, sizeof(int64_t) * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_out, sizeof(double) * kInfo * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_inst, sizeof(BatchInst) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_order, sizeof(int) * 3 * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_counts, sizeof(int) * 5);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_lock, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMemset(S->d_lock, 0, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_shift, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_out, sizeof(double) * kInfo * maxa);
    S->payload_stride = (6 * cfg->max_m * cfg->max_q + 2 * cfg->max_m + cfg->max_q + 3) / 4 * 4;
    if (e == cudaSuccess) e = cudaMalloc(&S->d_stepids, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_stepids, sizeof(int) * maxa);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_payload, sizeof(float) * (size_t)maxa * S->payload_stride);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_payload, sizeof(float) * (size_t)maxa * S->payload_stride);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    for (cudaEvent_t &ev : S->ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMemset(S->d_out, 0, sizeof(double) * kInfo * maxa);
    if (e != cudaSuccess)
        return bail(e == cudaErrorMemoryAllocation ? ADMM_ENOMEM : ADMM_ECUDA, cudaGetErrorString(e));
    std::memset(S->h_inst, 0, sizeof(BatchInst) * maxa);
    // launch shape of a tick: kernel and slices for the configured max m, q
    S->mbound = batch_mbound(cfg->max_m);
    S->slice = batch_slice_doubles(cfg->max_m, cfg->max_q);
    const BatchSmem bs = batch_cta_smem(cfg->max_m, cfg->max_q, cfg->batch.warps_per_cta,
                                        std::max(1, cfg->batch.cluster_size), cfg->batch.small_max_elements > 0,
                                        S->slice);
    S->smem = bs.bytes;
    S->stage_off = bs.stage_off;
    const int per_sm = batch_blocks_per_sm(cfg->batch.warps_per_cta, S->mbound, S->smem);
    if (per_sm < 1) return bail(ADMM_EUNSUPPORTED, "tick kernel cannot be resident");
    const int use = cfg->batch.ctas_per_sm > 0 ? std::min(cfg->batch.ctas_per_sm, per_sm) : per_sm;
    S->cluster = cfg->batch.cluster_size > 1 ? cfg->batch.cluster_size : 1;
    if (S->cluster > 1) {
        const int nc = batch_max_clusters(cfg->batch.warps_per_cta, S->mbound, S->cluster, S->smem);
        if (nc < 1) return bail(ADMM_EUNSUPPORTED, "clusters of this size cannot be resident");
        S->grid = std::max(1, std::min(nc, S->nsm * use / S->cluster)) * S->cluster;
    } else {
        S->grid = S->nsm * use;
    }
    // capture the tick: reset queue heads, run tick_iters iterations of every active instance
    BatchArgs a{};
    a.inst = S->d_inst;
    a.orderX = S->d_order;
    a.orderL = S->d_order + maxa;
    a.orderS = S->d_order + 2 * maxa;
    a.nLS = S->d_counts;
    a.qX = S->d_q;
    a.qL = S->d_q + 1;
    a.qS = S->d_q + 2;
    S->store.fill_args(a);
    a.f0 = S->store.f0;
    a.out = S->d_out;
    a.slice_doubles = (int)S->slice;
    a.stage_off = S->stage_off;
    a.iter_budget = cfg->tick_iters;
    a.tick_work = (const float *)(S->d_counts + 3);
    a.tick_rounds = S->d_counts + 4;
    a.lock = S->d_lock;
    a.r_tol = stop_r_tol(prm->precision, prm->r_tol);
    a.s_tol = stop_s_tol(prm->precision, prm->s_tol);
    a.adapt_target = prm->r_tol / prm->s_tol;
    a.adapt_start = prm->adapt_start;
    a.tau = prm->tau;
    a.max_iter = prm->max_iter;
    a.check_every = prm->check_every;
    a.xmin_mode = prm->xmin_mode;
    a.sweep = prm->sweep;
    a.adapt = prm->adapt_rho;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(S->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_q, 0, 3 * sizeof(int), S->st);
    if (e == cudaSuccess)
        e = launch_batch(cfg->batch.warps_per_cta, S->mbound, S->grid, S->cluster, a, S->smem, false, S->st);
    cudaError_t e2 = cudaStreamEndCapture(S->st, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&S->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return bail(ADMM_ECUDA, std::string("tick graph: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    S->active.assign(maxa, nullptr);
    for (int s = maxa - 1; s >= 0; --s) S->free_slots.push_back(s);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return ADMM_OK;
}

admm_status admm_server_submit(admm_server *S, const admm_problem *P, int64_t session, int64_t *ticket)
{
    clear_last_error();
    if (!S || !P || !ticket) return sfail(ADMM_EINVAL, "NULL argument");
    if (P->on_device) return sfail(ADMM_EINVAL, "server requests take host arrays (on_device = 0)");
    if (P->m > S->cfg.max_m || P->q > S->cfg.max_q)
        return sfail(ADMM_EUNSUPPORTED, "instance exceeds the server's max_m or max_q");
    auto r = std::make_shared<Request>();
    r->t_submit = now_s();
    std::string why;
    if (!stage_instance(*P, r->staged, why)) return sfail(ADMM_EINVAL, "invalid problem: " + why);
    const InstSizes z = inst_sizes(P->n, P->m, P->q);
    if (z.e > S->cfg.store_elements) return sfail(ADMM_EUNSUPPORTED, "instance larger than the device store");
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    r->session = session;
    if (session >= 0) S->sessions[session]; // creates the session record
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return ADMM_OK;
}

admm_status admm_server_submit_step(admm_server *S, int64_t session, const admm_step *st, int64_t *ticket)
{
    clear_last_error();
    if (!S || !st || !ticket || session < 0) return sfail(ADMM_EINVAL, "bad argument");
    const int m = st->m, q = st->q, mq = m * q;
    if (m < 1 || q < 1 || m > S->cfg.max_m || q > S->cfg.max_q) return sfail(ADMM_EINVAL, "bad step shape");
    const double *arrs[9] = {st->f2, st->f1, st->f0, st->g2, st->g1, st->g0, st->x_lo, st->x_hi, st->y};
    for (const double *a : arrs)
        if (!a) return sfail(ADMM_EINVAL, "a step array is NULL");
    auto r = std::make_shared<Request>();
    r->t_submit = now_s();
    r->is_step = true;
    r->step_m = m;
    r->step_q = q;
    r->payload.resize((size_t)6 * mq + 2 * m + q);
    for (int t = 0; t < 6; ++t)
        for (int u = 0; u < mq; ++u) {
            const double v = arrs[t][u];
            if (!std::isfinite(v)) return sfail(ADMM_EINVAL, "non-finite step coefficient");
            if ((t == 0 || t == 3) && v < 0.0) return sfail(ADMM_EINVAL, "f2 < 0 or g2 < 0 in the step");
            r->payload[(size_t)t * mq + u] = (float)v;
        }
    for (int i = 0; i < m; ++i) {
        if (!std::isfinite(st->x_lo[i]) || !std::isfinite(st->x_hi[i]) || st->x_lo[i] > st->x_hi[i])
            return sfail(ADMM_EINVAL, "bad step bounds");
        r->payload[(size_t)6 * mq + i] = (float)st->x_lo[i];
        r->payload[(size_t)6 * mq + m + i] = (float)st->x_hi[i];
    }
    for (int j = 0; j < q; ++j) {
        if (!std::isfinite(st->y[j])) return sfail(ADMM_EINVAL, "non-finite step demand");
        r->payload[(size_t)6 * mq + 2 * m + j] = (float)st->y[j];
    }
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    r->session = session;
    S->sessions[session];
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return ADMM_OK;
}

admm_status admm_server_cancel(admm_server *S, int64_t ticket)
{
    clear_last_error();
    if (!S) return sfail(ADMM_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return sfail(ADMM_EINVAL, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (r->done) return ADMM_OK;
    r->cancel = true;
    auto q = std::find(S->pending.begin(), S->pending.end(), r);
    if (q != S->pending.end()) { // not admitted yet
        S->pending.erase(q);
        r->status = ADMM_ECANCELLED;
        r->t_finish = now_s();
        r->done = true;
        S->cv_done.notify_all();
    }
    return ADMM_OK;
}

admm_status admm_server_poll(admm_server *S, int64_t ticket, int32_t wait_ms, admm_result *out, double *times)
{
    clear_last_error();
    if (!S) return sfail(ADMM_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return sfail(ADMM_EINVAL, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (!r->done && wait_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return r->done; });
    if (!r->done) return ADMM_EPENDING;
    S->reqs.erase(it);
    lk.unlock();
    if (times) {
        times[0] = r->t_admit > 0 ? r->t_admit - r->t_submit : -1.0;
        times[1] = r->t_finish - r->t_submit;
        times[2] = r->warm ? 1.0 : 0.0;
    }
    if (out) {
        out->iters = (int32_t)r->info[0];
        out->converged = r->info[1] != 0.0;
        out->r = r->info[2];
        out->sigma = r->info[3];
        out->objective = r->info[11];
        out->status = r->status;
        if (out->x && !r->x.empty()) std::memcpy(out->x, r->x.data(), sizeof(double) * r->x.size());
        if (out->x1 && !r->x1.empty()) std::memcpy(out->x1, r->x1.data(), sizeof(double) * r->x1.size());
    }
    return r->status == ADMM_ENOTCONVERGED ? ADMM_OK : r->status;
}

admm_status admm_server_drain(admm_server *S, int32_t max, int64_t *tickets, double *latency_s, int32_t *iters,
                              int32_t *status, int32_t *count)
{
    if (!S || !count || max < 0 || (max > 0 && (!tickets || !latency_s || !iters || !status)))
        return sfail(ADMM_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int k = 0;
    for (auto it = S->reqs.begin(); it != S->reqs.end() && k < max;) {
        const std::shared_ptr<Request> &r = it->second;
        if (!r->done) {
            ++it;
            continue;
        }
        tickets[k] = r->ticket;
        latency_s[k] = r->t_finish - r->t_submit;
        iters[k] = (int32_t)r->info[0];
        status[k] = (int32_t)r->status;
        ++k;
        it = S->reqs.erase(it);
    }
    *count = k;
    return ADMM_OK;
}

admm_status admm_server_stats(admm_server *S, double *stats, int32_t count)
{
    if (!S || !stats || count < 1) return sfail(ADMM_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    double v[10] = {S->stats[0], S->stats[1], S->stats[2], 0.0, (double)S->pending.size(), 0.0, 0.0, S->stats[3],
                    S->stats[4], S->stats[5]};
    for (auto &p : S->active)
        if (p) v[3] += 1;
    v[5] = (double)S->store.ae.free_total() / (double)std::max<int64_t>(1, S->store.ae.capacity());
    v[6] = (double)S->sessions.size();
    for (int t = 0; t < count && t < 10; ++t) stats[t] = v[t];
    return ADMM_OK;
}

admm_status admm_server_destroy(admm_server *S)
{
    if (!S) return ADMM_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->exec) cudaGraphExecDestroy(S->exec);
    S->store.free_all();
    void *d[] = {S->d_inst,  S->d_order, S->d_counts,  S->d_q,    S->d_shift, S->d_out,
                     S->d_tmp,   S->d_stepids, S->d_payload, S->d_gids, S->d_goff, S->d_lock};
    for (void *p : d)
        if (p) cudaFree(p);
    void *h[] = {S->h_inst,  S->h_order,   S->h_counts, S->h_shift, S->h_out,
                     S->pinned,  S->h_stepids, S->h_payload, S->h_gids, S->h_goff, S->h_gather};
    for (void *p : h)
        if (p) cudaFreeHost(p);
    if (S->st) cudaStreamDestroy(S->st);
    for (cudaEvent_t ev : S->ev)
        if (ev) cudaEventDestroy(ev);
    delete S;
    return ADMM_OK;
}

} // extern "C"

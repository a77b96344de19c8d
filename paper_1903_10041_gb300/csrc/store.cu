// Device store of many instances (see store.h).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "store.h"

namespace admm_impl {

void RangeAlloc::init(int64_t cap)
{
    cap_ = cap;
    free_.clear();
    if (cap > 0) free_[0] = cap;
}

int64_t RangeAlloc::alloc(int64_t len, int64_t align)
{
    if (len <= 0) return 0;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        const int64_t start = it->first, flen = it->second;
        const int64_t a = (start + align - 1) / align * align;
        if (a + len > start + flen) continue;
        free_.erase(it);
        if (a > start) free_[start] = a - start;
        if (a + len < start + flen) free_[a + len] = start + flen - (a + len);
        return a;
    }
    return -1;
}

void RangeAlloc::release(int64_t off, int64_t len)
{
    if (len <= 0) return;
    auto next = free_.lower_bound(off);
    if (next != free_.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            off = prev->first;
            len += prev->second;
            free_.erase(prev);
        }
    }
    next = free_.lower_bound(off);
    if (next != free_.end() && off + len == next->first) {
        len += next->second;
        free_.erase(next);
    }
    free_[off] = len;
}

int64_t RangeAlloc::free_total() const
{
    int64_t t = 0;
    for (auto &kv : free_) t += kv.second;
    return t;
}

int64_t RangeAlloc::largest_free() const
{
    int64_t t = 0;
    for (auto &kv : free_) t = std::max(t, kv.second);
    return t;
}

InstSizes inst_sizes(int n, int m, int q)
{
    const int64_t ld = (n + 3) / 4 * 4;
    return {(int64_t)m * q * ld, (int64_t)m * ld, (int64_t)q * ld, (int64_t)m * q, (int64_t)scal_size(m, q), m};
}

bool stage_instance(const admm_problem &P, Staged &S, std::string &why)
{
    const int n = P.n, m = P.m, q = P.q;
    if (n < 1 || m < 1 || q < 1) {
        why = "n, m, q must be >= 1";
        return false;
    }
    const int ld = (n + 3) / 4 * 4;
    S.n = n;
    S.m = m;
    S.q = q;
    S.ld = ld;
    if (P.coef_shared != 0 && P.coef_shared != 1) {
        why = "coef_shared must be 0 or 1";
        return false;
    }
    S.cs = P.coef_shared;
    const size_t ne = (size_t)m * q * ld, nb = (size_t)m * ld, nc = (size_t)q * ld;
    for (auto &v : S.e) v.assign(ne, 0.0f);
    for (auto &v : S.b) v.assign(nb, 0.0f);
    S.y.assign(nc, 0.0f);
    S.sumg0.assign((size_t)m * q, 0.0);
    S.c.assign(P.c, P.c + m);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < n; ++k) {
            const double a = P.x_lo[(size_t)i * n + k], b = P.x_hi[(size_t)i * n + k];
            if (!std::isfinite(a) || !std::isfinite(b)) {
                why = "non-finite bound";
                return false;
            }
            if (a > b) {
                why = "x_lo > x_hi";
                return false;
            }
            S.b[0][(size_t)i * ld + k] = (float)a;
            S.b[1][(size_t)i * ld + k] = (float)b;
        }
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k) {
            const double v = P.y[(size_t)j * n + k];
            if (!std::isfinite(v)) {
                why = "non-finite demand";
                return false;
            }
            S.y[(size_t)j * ld + k] = (float)v;
        }
    const double *src[6] = {P.f2, P.f1, P.f0, P.g2, P.g1, P.g0};
    for (int i = 0; i < m; ++i) {
        if (std::isnan(S.c[i])) {
            why = "c is NaN";
            return false;
        }
        for (int j = 0; j < q; ++j) {
            double s0 = 0.0, smin = 0.0;
            for (int k = 0; k < n; ++k) {
                // scenario-shared maps: read once per source and stored in every
                // scenario's row (the batched kernel indexes coefficients like x)
                const size_t e = (S.cs ? (size_t)i : (size_t)i * q + j) * n + k;
                const size_t d = ((size_t)i * q + j) * ld + k, dc = d;
                double v[6];
                for (int t = 0; t < 6; ++t) {
                    v[t] = src[t][e];
                    if (!std::isfinite(v[t])) {
                        why = "non-finite coefficient";
                        return false;
                    }
                    S.e[t][dc] = (float)v[t];
                }
                if (v[0] < 0.0 || v[3] < 0.0) {
                    why = "f2 < 0 or g2 < 0 (Assumption 1 needs convex f, g)";
                    return false;
                }
                const double l = P.x_lo[(size_t)i * n + k], h = P.x_hi[(size_t)i * n + k];
                double xm = v[3] > 0.0 ? -v[4] / (2.0 * v[3]) : (v[4] > 0.0 ? l : h);
                xm = std::min(std::max(xm, l), h);
                s0 += v[5];
                smin += v[3] * xm * xm + v[4] * xm + v[5];
                const float lf = S.b[0][(size_t)i * ld + k], hf = S.b[1][(size_t)i * ld + k];
                S.e[6][d] = 0.0f < lf ? lf : (0.0f > hf ? hf : 0.0f);
            }
            S.sumg0[(size_t)i * q + j] = s0;
            if (smin > S.c[i] * (1.0 + 1e-12) + 1e-12) {
                why = "sum_k min g > c for some (i, j): infeasible";
                return false;
            }
        }
    }
    return true;
}

cudaError_t Store::allocate(int64_t e, int64_t b, int64_t c_, int64_t p, int64_t s_, int64_t m)
{
    cap_e = e;
    cap_b = b;
    cap_c = c_;
    cap_p = p;
    cap_s = s_;
    cap_m = m;
    float **fe[7] = {&f2, &f1, &f0, &g2, &g1, &g0, &x};
    for (float **a : fe) {
        cudaError_t r = cudaMalloc(a, sizeof(float) * std::max<int64_t>(e, 4));
        if (r != cudaSuccess) return r;
    }
    float **fb[2] = {&lo, &hi};
    for (float **a : fb) {
        cudaError_t r = cudaMalloc(a, sizeof(float) * std::max<int64_t>(b, 4));
        if (r != cudaSuccess) return r;
    }
    float **fc[5] = {&y, &s, &s_lo, &mu, &mu_lo};
    for (float **a : fc) {
        cudaError_t r = cudaMalloc(a, sizeof(float) * std::max<int64_t>(c_, 4));
        if (r != cudaSuccess) return r;
    }
    cudaError_t r = cudaMalloc(&sumg0, sizeof(double) * std::max<int64_t>(p, 1));
    if (r == cudaSuccess) r = cudaMalloc(&scal, sizeof(double) * std::max<int64_t>(s_, 1));
    if (r == cudaSuccess) r = cudaMalloc(&c, sizeof(double) * std::max<int64_t>(m, 1));
    if (r != cudaSuccess) return r;
    ae.init(e);
    ab.init(b);
    ac.init(c_);
    ap.init(p);
    as.init(s_);
    am.init(m);
    return cudaSuccess;
}

void Store::free_all()
{
    void *all[] = {f2, f1, f0, g2, g1, g0, x, lo, hi, y, s, s_lo, mu, mu_lo, sumg0, scal, c};
    for (void *p : all)
        if (p) cudaFree(p);
    f2 = f1 = f0 = g2 = g1 = g0 = x = lo = hi = y = s = s_lo = mu = mu_lo = nullptr;
    sumg0 = scal = c = nullptr;
}

bool Store::place(int n, int m, int q, BatchInst &I)
{
    const InstSizes z = inst_sizes(n, m, q);
    const int64_t oe = ae.alloc(z.e, 4);
    const int64_t ob = oe < 0 ? -1 : ab.alloc(z.b, 4);
    const int64_t oc = ob < 0 ? -1 : ac.alloc(z.c, 4);
    const int64_t op = oc < 0 ? -1 : ap.alloc(z.p, 1);
    const int64_t os = op < 0 ? -1 : as.alloc(z.s, 1);
    const int64_t om = os < 0 ? -1 : am.alloc(z.m, 1);
    if (om < 0) {
        if (oe >= 0) ae.release(oe, z.e);
        if (ob >= 0) ab.release(ob, z.b);
        if (oc >= 0) ac.release(oc, z.c);
        if (op >= 0) ap.release(op, z.p);
        if (os >= 0) as.release(os, z.s);
        return false;
    }
    I.n = n;
    I.m = m;
    I.q = q;
    I.ld = (n + 3) / 4 * 4;
    I.off_e = oe;
    I.off_b = ob;
    I.off_c = oc;
    I.off_pair = (int)op;
    I.off_scal = (int)os;
    I.off_src = (int)om;
    I.cs = 0;
    return true;
}

void Store::release(const BatchInst &I)
{
    const InstSizes z = inst_sizes(I.n, I.m, I.q);
    ae.release(I.off_e, z.e);
    ab.release(I.off_b, z.b);
    ac.release(I.off_c, z.c);
    ap.release(I.off_pair, z.p);
    as.release(I.off_scal, z.s);
    am.release(I.off_src, z.m);
}

cudaError_t Store::upload(const BatchInst &I, const Staged &S, const admm_params &prm, float *pinned, size_t pinned_n,
                          cudaStream_t st)
{
    const InstSizes z = inst_sizes(I.n, I.m, I.q);
    const size_t need = 7 * (size_t)z.e + 2 * (size_t)z.b + (size_t)z.c;
    if (need > pinned_n) return cudaErrorInvalidValue;
    float *dst_e[7] = {f2, f1, f0, g2, g1, g0, x};
    size_t at = 0;
    cudaError_t r = cudaStreamSynchronize(st); // the staging buffer may still be in use
    if (r != cudaSuccess) return r;
    for (int t = 0; t < 7; ++t) {
        std::memcpy(pinned + at, S.e[t].data(), sizeof(float) * z.e);
        r = cudaMemcpyAsync(dst_e[t] + I.off_e, pinned + at, sizeof(float) * z.e, cudaMemcpyHostToDevice, st);
        if (r != cudaSuccess) return r;
        at += z.e;
    }
    float *dst_b[2] = {lo, hi};
    for (int t = 0; t < 2; ++t) {
        std::memcpy(pinned + at, S.b[t].data(), sizeof(float) * z.b);
        r = cudaMemcpyAsync(dst_b[t] + I.off_b, pinned + at, sizeof(float) * z.b, cudaMemcpyHostToDevice, st);
        if (r != cudaSuccess) return r;
        at += z.b;
    }
    std::memcpy(pinned + at, S.y.data(), sizeof(float) * z.c);
    r = cudaMemcpyAsync(y + I.off_c, pinned + at, sizeof(float) * z.c, cudaMemcpyHostToDevice, st);
    if (r != cudaSuccess) return r;
    float *zc[4] = {s, s_lo, mu, mu_lo};
    for (float *a : zc) {
        r = cudaMemsetAsync(a + I.off_c, 0, sizeof(float) * z.c, st);
        if (r != cudaSuccess) return r;
    }
    r = cudaMemcpyAsync(sumg0 + I.off_pair, S.sumg0.data(), sizeof(double) * z.p, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(c + I.off_src, S.c.data(), sizeof(double) * z.m, cudaMemcpyHostToDevice, st);
    std::vector<double> sc(z.s, 0.0);
    const int mq = I.m * I.q;
    for (int t = 0; t < 4; ++t) sc[5 * mq + I.m + t] = prm.rho[t];
    if (prm.rho2_over_n) sc[5 * mq + I.m + 1] = prm.rho[1] / (double)I.n;
    sc[5 * mq + I.m + 4] = 1.0;
    sc[5 * mq + I.m + 5] = 1.0;
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(scal + I.off_scal, sc.data(), sizeof(double) * z.s, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    return r;
}

void Store::fill_args(BatchArgs &a) const
{
    a.f2 = f2;
    a.f1 = f1;
    a.f0 = f0;
    a.g2 = g2;
    a.g1 = g1;
    a.g0 = g0;
    a.lo = lo;
    a.hi = hi;
    a.y = y;
    a.x = x;
    a.s = s;
    a.s_lo = s_lo;
    a.mu = mu;
    a.mu_lo = mu_lo;
    a.c = c;
    a.sumg0 = sumg0;
    a.scal = scal;
}

cudaError_t store_get_state(const Store &S, const BatchInst &I, admm_state *o, double *tmp, cudaStream_t st)
{
    const int n = I.n, m = I.m, q = I.q, mq = m * q;
    const bool dev = o->on_device != 0;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t r = cudaSuccess;
    if (o->x) {
        convert_rows_f32_to_f64(tmp, n, S.x + I.off_e, I.ld, n, mq, st);
        r = cudaMemcpyAsync(o->x, tmp, sizeof(double) * mq * n, k, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (r != cudaSuccess) return r;
    }
    if (o->s) {
        convert_rows_ff_to_f64(tmp, n, S.s + I.off_c, S.s_lo + I.off_c, I.ld, n, q, st);
        r = cudaMemcpyAsync(o->s, tmp, sizeof(double) * q * n, k, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (r != cudaSuccess) return r;
    }
    if (o->mu) {
        convert_rows_ff_to_f64(tmp, n, S.mu + I.off_c, S.mu_lo + I.off_c, I.ld, n, q, st);
        r = cudaMemcpyAsync(o->mu, tmp, sizeof(double) * q * n, k, st);
        if (r == cudaSuccess) r = cudaStreamSynchronize(st);
        if (r != cudaSuccess) return r;
    }
    double *pairs[5] = {o->lam, o->zeta, o->h, o->p, o->nu};
    for (int t = 0; t < 5 && r == cudaSuccess; ++t)
        if (pairs[t]) r = cudaMemcpyAsync(pairs[t], S.scal + I.off_scal + (size_t)t * mq, sizeof(double) * mq, k, st);
    if (r == cudaSuccess && o->x1) r = cudaMemcpyAsync(o->x1, S.scal + I.off_scal + 5 * mq, sizeof(double) * m, k, st);
    double tail[6];
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(tail, S.scal + I.off_scal + 5 * mq + m, sizeof tail, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    if (r != cudaSuccess) return r;
    for (int t = 0; t < 4; ++t) o->rho[t] = tail[t];
    o->cold = tail[4] != 0.0;
    return cudaSuccess;
}

cudaError_t store_set_state(const Store &S, const BatchInst &I, const admm_state *w, double *tmp, cudaStream_t st)
{
    const int n = I.n, m = I.m, q = I.q, mq = m * q;
    const bool dev = w->on_device != 0;
    const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t r = cudaMemcpyAsync(tmp, w->x, sizeof(double) * mq * n, k, st);
    if (r != cudaSuccess) return r;
    convert_rows_f64_to_f32(S.x + I.off_e, I.ld, tmp, n, n, mq, st);
    r = cudaStreamSynchronize(st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(tmp, w->s, sizeof(double) * q * n, k, st);
    if (r != cudaSuccess) return r;
    split_rows_f64_to_ff(S.s + I.off_c, S.s_lo + I.off_c, I.ld, tmp, n, n, q, st);
    r = cudaStreamSynchronize(st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(tmp, w->mu, sizeof(double) * q * n, k, st);
    if (r != cudaSuccess) return r;
    split_rows_f64_to_ff(S.mu + I.off_c, S.mu_lo + I.off_c, I.ld, tmp, n, n, q, st);
    r = cudaStreamSynchronize(st);
    const double *pairs[5] = {w->lam, w->zeta, w->h, w->p, w->nu};
    for (int t = 0; t < 5 && r == cudaSuccess; ++t)
        r = cudaMemcpyAsync(S.scal + I.off_scal + (size_t)t * mq, pairs[t], sizeof(double) * mq, k, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(S.scal + I.off_scal + 5 * mq, w->x1, sizeof(double) * m, k, st);
    double tail[6] = {w->rho[0], w->rho[1], w->rho[2], w->rho[3], w->cold ? 1.0 : 0.0, 1.0};
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(S.scal + I.off_scal + 5 * mq + m, tail, sizeof tail, cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    return r;
}

} // namespace admm_impl

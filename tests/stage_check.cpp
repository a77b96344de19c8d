// Check of the batched path's host-side staging (validation and FP32
// packing of one instance, store.h) on a small problem: layout [m][q][ld]
// with ld = n rounded up to 4 and zero padding, the FP32 values, the FP64
// sums of beta_0 per (i, j), the start x = clamp(0, lo, hi), and each kind
// of invalid data refused with a message.  Links libadmm.so; needs no GPU.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "store.h"

using admm_impl::Staged;
using admm_impl::stage_instance;

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            std::fprintf(stderr, "check failed line %d: %s\n", __LINE__, #c); \
            return 1;                                                   \
        }                                                               \
    } while (0)

struct Data {
    int n = 7, m = 2, q = 3;
    std::vector<double> a[6], lo, hi, y, c;
    Data()
    {
        const size_t ne = (size_t)m * q * n;
        for (int t = 0; t < 6; ++t) {
            a[t].resize(ne);
            for (size_t e = 0; e < ne; ++e) a[t][e] = 0.01 * (double)((e * 7 + t * 13) % 17) + (t == 3 ? 0.05 : 0.0);
        }
        lo.assign((size_t)m * n, -1.0);
        hi.assign((size_t)m * n, 2.0);
        lo[3] = 0.5;   // 0 below the interval: the start is lo
        hi[9] = -0.25; // 0 above the interval: the start is hi
        lo[9] = -0.75;
        y.resize((size_t)q * n);
        for (size_t t = 0; t < y.size(); ++t) y[t] = 0.5 + 0.1 * (double)(t % 5);
        c.assign(m, 1e9);
    }
    admm_problem prob() const
    {
        admm_problem P{};
        P.n = n; P.m = m; P.q = q;
        P.f2 = a[0].data(); P.f1 = a[1].data(); P.f0 = a[2].data();
        P.g2 = a[3].data(); P.g1 = a[4].data(); P.g0 = a[5].data();
        P.x_lo = lo.data(); P.x_hi = hi.data(); P.y = y.data(); P.c = c.data();
        return P;
    }
};

static bool refused(const Data &d, const char *what)
{
    Staged S;
    std::string why;
    const bool ok = stage_instance(d.prob(), S, why);
    if (ok || why.empty()) std::fprintf(stderr, "%s was not refused\n", what);
    return !ok && !why.empty();
}

int main()
{
    Data d;
    Staged S;
    std::string why;
    CHECK(stage_instance(d.prob(), S, why));
    const int n = d.n, m = d.m, q = d.q, ld = 8;
    CHECK(S.ld == ld && S.n == n && S.m == m && S.q == q);
    for (int t = 0; t < 6; ++t) CHECK(S.e[t].size() == (size_t)m * q * ld);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double s0 = 0.0;
            for (int k = 0; k < ld; ++k) {
                const size_t dst = ((size_t)i * q + j) * ld + k;
                if (k >= n) { // padding
                    for (int t = 0; t < 7; ++t) CHECK(S.e[t][dst] == 0.0f);
                    continue;
                }
                const size_t src = ((size_t)i * q + j) * n + k;
                for (int t = 0; t < 6; ++t) CHECK(S.e[t][dst] == (float)d.a[t][src]);
                const double l = d.lo[(size_t)i * n + k], h = d.hi[(size_t)i * n + k];
                CHECK(S.e[6][dst] == (float)(0.0 < l ? l : (0.0 > h ? h : 0.0)));
                s0 += d.a[5][src];
            }
            CHECK(S.sumg0[(size_t)i * q + j] == s0);
        }
    CHECK(S.e[6][(size_t)(0 * q + 1) * ld + 3] == 0.5f && S.e[6][(size_t)(1 * q + 2) * ld + 2] == -0.25f);
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < ld; ++k)
            CHECK(S.y[(size_t)j * ld + k] == (k < n ? (float)d.y[(size_t)j * n + k] : 0.0f));

    { Data b; b.a[1][5] = NAN; CHECK(refused(b, "a NaN coefficient")); }
    { Data b; b.a[0][4] = -0.1; CHECK(refused(b, "f2 < 0")); }
    { Data b; b.a[3][8] = -0.1; CHECK(refused(b, "g2 < 0")); }
    { Data b; b.lo[2] = 3.0; CHECK(refused(b, "lo > hi")); }
    { Data b; b.hi[1] = INFINITY; CHECK(refused(b, "an infinite bound")); }
    { Data b; b.y[4] = NAN; CHECK(refused(b, "a NaN demand")); }
    { Data b; b.c[1] = NAN; CHECK(refused(b, "a NaN capacity")); }
    { Data b; b.c[0] = -100.0; CHECK(refused(b, "a capacity below the least possible loss")); }
    { Data b; b.n = 0; CHECK(refused(b, "an empty horizon")); }
    std::printf("staging ok\n");
    return 0;
}

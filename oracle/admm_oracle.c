/*
 * FP64 CPU oracle of the parallel ADMM solver for robust quadratic resource
 * allocation (Qureshi, East, Cannon: "Parallel ADMM for robust quadratic
 * optimal resource allocation problems").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the solver library never does.
 * It shares no code, header or constant with the CUDA path.
 *
 * What it computes, in the paper's order and notation:
 *   - Algorithm 1 (Sec. III-B): the minimiser of A x^4 + B x^3 + C x^2 + D x
 *     through the closed-form roots of the monic cubic x^3 + b x^2 + c x + d.
 *   - The ADMM iteration (a)-(i) of App. A on the reformulation (admm_opt),
 *     with dense arrays x, z, lambda [m][q][n]; s, mu [q][n]; h, p, nu [m][q];
 *     x_1 [m].  Step (a) uses the (theta, phi) form given after the
 *     iteration.
 *   - The residuals r and sigma of App. A and the stop test of Alg. 2 step 3
 *     (r < r-bar and sigma < sigma-bar), checked every `check_every`
 *     iterations as in Sec. IV-B.
 *   - The objective (1/q) sum f of eq. (2) and a KKT residual of eq. (2).
 *
 * Readings of points the paper leaves open, numbered R1..R14 wherever they are cited:
 *   R1  step (c) averages: x_1^(i) = (1/q) sum_j (x_1^(i,j) - nu^(i,j)).
 *   R2  theta_k^(i,j) = z_k^(i,j) + lambda_k^(i,j) (the paper prints
 *       lambda_k^(i)); y in L is y^(j).
 *   R3  step (a) takes the constrained minimiser: with two local minima,
 *       both roots are clamped to the bounds and the better clamped value is
 *       kept ("exact").  The literal Pi(argmin) is mode "paper".
 *   R4  a tie delta-f = 0 keeps x_1 (the smaller root), as Algorithm 1's else
 *       branch does.
 *   R5  A = 0 (beta_2 = 0): the quadratic C x^2 + D x is minimised directly.
 *   R6  Algorithm 1 numerics: acos argument clamped to [-1, 1]; real cube
 *       roots; the stable Cardano pair S = cbrt(R + sgn(R) sqrt(Delta)),
 *       T = -Q / S (same values as the printed S, T); exact comparisons for
 *       Delta > 0 and Q = R = 0.
 *   R7  step (a) sweeps the sources i = 1..m in order, each using the newest
 *       x^(l), l < i (Gauss-Seidel); "jacobi" uses the previous iterate.
 *   R8  initial values are zero (x clamped to its bounds).
 *   R10 sigma is taken as printed, with the max over (i, j) and the tilde
 *       meaning the previous iterate.
 *
 * Compiled with -O2 -ffp-contract=off (no fast-math), so that x86 and Arm
 * give the same rounding apart from libm.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n, m, q;
    const double *f2, *f1, *f0; /* alpha_{k,2..0}^{(i,j)}  [m][q][n] */
    const double *g2, *g1, *g0; /* beta_{k,2..0}^{(i,j)}   [m][q][n] */
    const double *lo, *hi;      /* bounds on x_k^{(i)}     [m][n]    */
    const double *y;            /* demand y_k^{(j)}        [q][n]    */
    const double *c;            /* capacity c^{(i)}        [m]       */
} orc_problem;

typedef struct {
    double rho1, rho2, rho3, rho4;
    double r_tol, s_tol;
    int max_iter, check_every;
    int xmin_mode; /* 0: exact (R3), 1: paper literal Pi(argmin) */
    int sweep;     /* 0: Gauss-Seidel over i (R7), 1: Jacobi */
    int threads;   /* OpenMP threads over columns; <= 0: 1 */
    int count_differs; /* also evaluate the other x-update mode and count disagreements */
    int adapt_rho;     /* Sec. IV-A: rescale rho_1..rho_4 by tau from the r / sigma ratio */
    double tau;
    int adapt_start;   /* the rescaling applies at check iterations t >= adapt_start (0: all) */
} orc_params;

typedef struct {
    double *x, *z, *lam; /* [m][q][n] */
    double *s, *mu;      /* [q][n] */
    double *h, *p, *nu;  /* [m][q] */
    double *x1;          /* [m] */
} orc_state;

typedef struct {
    int iters, converged;
    double r, sigma;
    double r_terms[4]; /* demand, z-g(x), h-1'z, x_1 copies */
    double s_terms[3]; /* rho1 z, rho2 h, rho3 s/x */
    long long branch_count[4]; /* Cardano, triple root, trig, quadratic */
    long long literal_differs; /* elements where "paper" and "exact" disagree */
    double rho[4];             /* penalties at exit (differ from the input with adapt_rho) */
} orc_report;

#define IDX3(i, j, k) ((((size_t)(i)) * q + (j)) * (size_t)n + (k))
#define IDX2(a, k) (((size_t)(a)) * (size_t)n + (k))

static double clampd(double v, double lo, double hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

/* delta-f of Algorithm 1: F(u) - F(v) for F(x) = x^4/4 + (b/3) x^3 + (c/2) x^2 + d x,
 * whose derivative is the monic cubic x^3 + b x^2 + c x + d. */
static double delta_f(double u, double v, double b, double c, double d)
{
    double u2 = u * u, v2 = v * v;
    return 0.25 * (u2 * u2 - v2 * v2) + (b / 3.0) * (u2 * u - v2 * v) + (c / 2.0) * (u2 - v2) + d * (u - v);
}

/* Roots of x^3 + b x^2 + c x + d (Sec. III-B).  Returns the number of
 * distinct formulas used: 1 (Delta > 0 or Q = R = 0) or 3 (trig), with the
 * roots in r[] and the branch id in *branch (0 Cardano, 1 triple, 2 trig). */
int orc_cubic_roots(double b, double c, double d, double *r, int *branch)
{
    double Q = c / 3.0 - b * b / 9.0;
    double R = b * c / 6.0 - b * b * b / 27.0 - d / 2.0;
    double Delta = Q * Q * Q + R * R;
    if (Delta > 0.0) {
        double sq = sqrt(Delta);
        double S = cbrt(R >= 0.0 ? R + sq : R - sq); /* R6: stable pair */
        double T = -Q / S;
        r[0] = S + T - b / 3.0;
        *branch = 0;
        return 1;
    }
    if (Q == 0.0 && R == 0.0) {
        r[0] = -b / 3.0; /* Vieta: triple root */
        *branch = 1;
        return 1;
    }
    {
        const double pi = 3.14159265358979323846;
        double arg = clampd(R / sqrt(-Q * Q * Q), -1.0, 1.0);
        double theta = acos(arg);
        double two_sq = 2.0 * sqrt(-Q);
        r[0] = two_sq * cos(theta / 3.0) - b / 3.0;                  /* x_a */
        r[1] = two_sq * cos(theta / 3.0 + 2.0 * pi / 3.0) - b / 3.0; /* x_b */
        r[2] = two_sq * cos(theta / 3.0 + 4.0 * pi / 3.0) - b / 3.0; /* x_c */
        *branch = 2;
        return 3;
    }
}

static void sort3(double *v)
{
    double t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

/* Algorithm 1 followed by the projection of step (a): minimiser of
 * A x^4 + B x^3 + C x^2 + D x over [lo, hi].  A >= 0; A = 0 needs C > 0. */
double orc_quartic_min(double A, double B, double C, double D, double lo, double hi,
                       int mode, int *branch_out)
{
    double r[3];
    int branch;
    if (A == 0.0) { /* R5 */
        if (branch_out) *branch_out = 3;
        return clampd(-D / (2.0 * C), lo, hi);
    }
    double b = 3.0 * B / (4.0 * A), c = C / (2.0 * A), d = D / (4.0 * A);
    int nr = orc_cubic_roots(b, c, d, r, &branch);
    if (branch_out) *branch_out = branch;
    if (nr == 1)
        return clampd(r[0], lo, hi);
    sort3(r); /* (x_1, x_2, x_3); x_2 is a maximiser and is dropped */
    if (mode == 1) {
        double xs = delta_f(r[0], r[2], b, c, d) > 0.0 ? r[2] : r[0];
        return clampd(xs, lo, hi);
    } else {
        double u = clampd(r[0], lo, hi), v = clampd(r[2], lo, hi);
        return delta_f(u, v, b, c, d) > 0.0 ? v : u; /* R4: tie keeps x_1 */
    }
}

/* Vectorised wrapper for tests. */
void orc_quartic_min_many(long long cnt, const double *A, const double *B, const double *C,
                          const double *D, const double *lo, const double *hi, int mode,
                          double *x, int *branch)
{
    for (long long t = 0; t < cnt; ++t)
        x[t] = orc_quartic_min(A[t], B[t], C[t], D[t], lo[t], hi[t], mode, branch ? &branch[t] : 0);
}

/* R8: x = Pi(0), every other variable zero. */
void orc_init_state(const orc_problem *P, orc_state *S)
{
    int n = P->n, m = P->m, q = P->q;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < n; ++k) {
                S->x[IDX3(i, j, k)] = clampd(0.0, P->lo[IDX2(i, k)], P->hi[IDX2(i, k)]);
                S->z[IDX3(i, j, k)] = 0.0;
                S->lam[IDX3(i, j, k)] = 0.0;
            }
    memset(S->s, 0, sizeof(double) * (size_t)q * n);
    memset(S->mu, 0, sizeof(double) * (size_t)q * n);
    memset(S->h, 0, sizeof(double) * (size_t)m * q);
    memset(S->p, 0, sizeof(double) * (size_t)m * q);
    memset(S->nu, 0, sizeof(double) * (size_t)m * q);
    memset(S->x1, 0, sizeof(double) * (size_t)m);
}

static double g_at(const orc_problem *P, size_t e, double x)
{
    return P->g2[e] * x * x + P->g1[e] * x + P->g0[e];
}

/* Coefficients of the step-(a) objective in x = x_k^{(i,j)} (theta, phi form):
 *   (1/q) f(x) + rho1/2 (theta - g(x))^2 + rho3/2 (phi - x)^2
 *   + [k = 1] rho4/2 (x_1^{(i)} + nu^{(i,j)} - x)^2
 * as A x^4 + B x^3 + C x^2 + D x + const. */
static void step_a_coeffs(const orc_problem *P, const orc_params *pr, size_t e, double theta,
                          double phi, int first, double psi, double *A, double *B, double *C,
                          double *D)
{
    double a2 = P->f2[e], a1 = P->f1[e];
    double b2 = P->g2[e], b1 = P->g1[e], b0 = P->g0[e];
    double w = b0 - theta; /* g(x) - theta = b2 x^2 + b1 x + w */
    double iq = 1.0 / (double)P->q;
    *A = 0.5 * pr->rho1 * b2 * b2;
    *B = 0.5 * pr->rho1 * 2.0 * b2 * b1;
    *C = a2 * iq + 0.5 * pr->rho1 * (b1 * b1 + 2.0 * b2 * w) + 0.5 * pr->rho3;
    *D = a1 * iq + 0.5 * pr->rho1 * 2.0 * b1 * w - pr->rho3 * phi;
    if (first) {
        *C += 0.5 * pr->rho4;
        *D -= pr->rho4 * psi;
    }
}

static double amax(double a, double b) { return a > b ? a : b; }

/* Step (a) of App. A on the columns of P: the x-update source by source;
 * for a fixed i the (j, k) updates are independent (Sec. II), so they may
 * run in any order.  k0 is the global index of P's first column (nonzero
 * only for a shard of columns, see orc_shard_phase_a): the copy term of
 * step (a) applies at global k = 0.  `xprev` holds x at the start of the
 * iteration (Jacobi sweep). */
static void step_a(const orc_problem *P, const orc_params *pr, orc_state *S, const double *xprev, int k0,
                   orc_report *rep)
{
    int n = P->n, m = P->m, q = P->q;
    long long differs = 0, br0 = 0, br1 = 0, br2 = 0, br3 = 0;
    for (int i = 0; i < m; ++i) {
#pragma omp parallel for collapse(2) reduction(+ : differs, br0, br1, br2, br3)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                const double *xs = (pr->sweep == 1) ? xprev : S->x;
                double others = 0.0;
                for (int l = 0; l < m; ++l)
                    if (l != i) others += xs[IDX3(l, j, k)];
                double theta = S->z[e] + S->lam[e];
                double phi = S->s[IDX2(j, k)] - others + P->y[IDX2(j, k)] + S->mu[IDX2(j, k)];
                double psi = S->x1[i] + S->nu[(size_t)i * q + j];
                double A, B, C, D;
                step_a_coeffs(P, pr, e, theta, phi, k + k0 == 0, psi, &A, &B, &C, &D);
                int br = 0;
                double lo = P->lo[IDX2(i, k)], hi = P->hi[IDX2(i, k)];
                double xn = orc_quartic_min(A, B, C, D, lo, hi, pr->xmin_mode, &br);
                if (pr->count_differs &&
                    orc_quartic_min(A, B, C, D, lo, hi, 1 - pr->xmin_mode, 0) != xn)
                    differs += 1;
                br0 += br == 0; br1 += br == 1; br2 += br == 2; br3 += br == 3;
                S->x[e] = xn;
            }
    }
    rep->literal_differs += differs;
    rep->branch_count[0] += br0; rep->branch_count[1] += br1;
    rep->branch_count[2] += br2; rep->branch_count[3] += br3;
}

/* Steps (e) and (f) on the columns of P (colsum receives sum_i x). */
static void steps_e_f(const orc_problem *P, orc_state *S, double *colsum)
{
    int n = P->n, m = P->m, q = P->q;
    /* (e) s-update: projection of sum_i x - y - mu onto [0, inf) */
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k) {
            double sx = 0.0;
            for (int i = 0; i < m; ++i)
                sx += S->x[IDX3(i, j, k)];
            colsum[IDX2(j, k)] = sx;
            double v = sx - P->y[IDX2(j, k)] - S->mu[IDX2(j, k)];
            S->s[IDX2(j, k)] = v > 0.0 ? v : 0.0;
        }
    /* (f) mu-update */
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k)
            S->mu[IDX2(j, k)] += S->s[IDX2(j, k)] - colsum[IDX2(j, k)] + P->y[IDX2(j, k)];
}

/* One ADMM iteration (a)-(i).  `xprev` holds x at the start of the iteration
 * (for Jacobi and the residuals).  Returns nothing; residuals are computed
 * by the caller from the saved previous iterate. */
static void admm_iteration(const orc_problem *P, const orc_params *pr, orc_state *S,
                           const double *xprev, double *gx, double *colsum, orc_report *rep)
{
    int n = P->n, m = P->m, q = P->q;

    /* (a) x-update */
    step_a(P, pr, S, xprev, 0, rep);
    for (size_t e = 0; e < (size_t)m * q * n; ++e)
        gx[e] = g_at(P, e, S->x[e]);

    double kappa = pr->rho2 / (pr->rho1 + (double)n * pr->rho2);
    /* (b) z-update: z = g(x) - lambda + kappa 1 (h + p - 1'(g(x) - lambda)) */
#pragma omp parallel for collapse(2)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double sum = 0.0;
            for (int k = 0; k < n; ++k)
                sum += gx[IDX3(i, j, k)] - S->lam[IDX3(i, j, k)];
            double t = kappa * (S->h[(size_t)i * q + j] + S->p[(size_t)i * q + j] - sum);
            for (int k = 0; k < n; ++k)
                S->z[IDX3(i, j, k)] = gx[IDX3(i, j, k)] - S->lam[IDX3(i, j, k)] + t;
        }
    /* (c) x_1-update (R1: the average over scenarios) */
    for (int i = 0; i < m; ++i) {
        double sum = 0.0;
        for (int j = 0; j < q; ++j)
            sum += S->x[IDX3(i, j, 0)] - S->nu[(size_t)i * q + j];
        S->x1[i] = sum / (double)q;
    }
    /* (d) h-update: projection of 1'z - p onto (-inf, c] */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double sz = 0.0;
            for (int k = 0; k < n; ++k)
                sz += S->z[IDX3(i, j, k)];
            double v = sz - S->p[(size_t)i * q + j];
            S->h[(size_t)i * q + j] = v < P->c[i] ? v : P->c[i];
        }
    /* (e), (f) */
    steps_e_f(P, S, colsum);
    /* (g) lambda-update */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < n; ++k)
                S->lam[IDX3(i, j, k)] += S->z[IDX3(i, j, k)] - gx[IDX3(i, j, k)];
    /* (h) nu-update */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j)
            S->nu[(size_t)i * q + j] += S->x1[i] - S->x[IDX3(i, j, 0)];
    /* (i) p-update */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double sz = 0.0;
            for (int k = 0; k < n; ++k)
                sz += S->z[IDX3(i, j, k)];
            S->p[(size_t)i * q + j] += S->h[(size_t)i * q + j] - sz;
        }
}

/* Primal and dual residuals of App. A at the current iterate, against the
 * previous iterate (xp, zp, sp, hp). */
static void residuals(const orc_problem *P, const orc_params *pr, const orc_state *S,
                      const double *gx, const double *xp, const double *zp, const double *sp,
                      const double *hp, orc_report *rep)
{
    int n = P->n, m = P->m, q = P->q;
    double r1 = 0, r2 = 0, r3 = 0, r4 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k) {
            double sx = 0.0, dx = 0.0;
            for (int i = 0; i < m; ++i) {
                sx += S->x[IDX3(i, j, k)];
                dx += S->x[IDX3(i, j, k)] - xp[IDX3(i, j, k)];
            }
            r1 = amax(r1, fabs(S->s[IDX2(j, k)] - sx + P->y[IDX2(j, k)]));
            s3 = amax(s3, fabs(S->s[IDX2(j, k)] - sp[IDX2(j, k)] - dx));
        }
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double sz = 0.0;
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                r2 = amax(r2, fabs(S->z[e] - gx[e]));
                s1 = amax(s1, fabs(S->z[e] - zp[e]));
                sz += S->z[e];
            }
            r3 = amax(r3, fabs(S->h[(size_t)i * q + j] - sz));
            r4 = amax(r4, fabs(S->x[IDX3(i, j, 0)] - S->x1[i]));
            s2 = amax(s2, fabs(S->h[(size_t)i * q + j] - hp[(size_t)i * q + j]));
        }
    rep->r_terms[0] = r1; rep->r_terms[1] = r2; rep->r_terms[2] = r3; rep->r_terms[3] = r4;
    rep->s_terms[0] = pr->rho1 * s1; rep->s_terms[1] = pr->rho2 * s2; rep->s_terms[2] = pr->rho3 * s3;
    rep->r = amax(amax(r1, r2), amax(r3, r4));
    rep->sigma = amax(amax(pr->rho1 * s1, pr->rho2 * s2), pr->rho3 * s3);
}

/* Run up to max_iter iterations from state S (updated in place).  Residuals
 * are evaluated after iteration t when t % check_every == 0 or t == max_iter;
 * the run stops at the first such t with r < r_tol and sigma < s_tol
 * (Alg. 2 step 3).  Returns 0 on success, -1 on allocation failure. */
int orc_solve(const orc_problem *P, const orc_params *pr_in, orc_state *S, orc_report *rep)
{
    int n = P->n, m = P->m, q = P->q;
    size_t ne = (size_t)m * q * n, nc = (size_t)q * n, np_ = (size_t)m * q;
    orc_params prm = *pr_in;
    const orc_params *pr = &prm;
    double *xp = malloc(sizeof(double) * ne), *zp = malloc(sizeof(double) * ne);
    double *gx = malloc(sizeof(double) * ne);
    double *sp = malloc(sizeof(double) * nc), *colsum = malloc(sizeof(double) * nc);
    double *hp = malloc(sizeof(double) * np_);
    memset(rep, 0, sizeof(*rep));
    if (!xp || !zp || !gx || !sp || !colsum || !hp) {
        free(xp); free(zp); free(gx); free(sp); free(colsum); free(hp);
        return -1;
    }
#ifdef _OPENMP
    omp_set_num_threads(pr->threads > 0 ? pr->threads : 1);
#endif
    rep->r = INFINITY;
    rep->sigma = INFINITY;
    for (int t = 1; t <= pr->max_iter; ++t) {
        memcpy(xp, S->x, sizeof(double) * ne);
        memcpy(zp, S->z, sizeof(double) * ne);
        memcpy(sp, S->s, sizeof(double) * nc);
        memcpy(hp, S->h, sizeof(double) * np_);
        admm_iteration(P, pr, S, xp, gx, colsum, rep);
        rep->iters = t;
        if (t % pr->check_every == 0 || t == pr->max_iter) {
            residuals(P, pr, S, gx, xp, zp, sp, hp, rep);
            if (rep->r < pr->r_tol && rep->sigma < pr->s_tol) {
                rep->converged = 1;
                break;
            }
            if (pr->adapt_rho && t < pr->max_iter && t >= pr->adapt_start) {
                /* Sec. IV-A: rho_i <- tau rho_i if r/sigma > 1.2 rbar/sbar,
                 * rho_i <- rho_i / tau if r/sigma < 0.8 rbar/sbar.  The scaled
                 * duals lambda, p, mu, nu carry a factor 1/rho and are rescaled
                 * by rho_old / rho_new (reading R11). */
                double ratio = rep->r / rep->sigma, target = pr->r_tol / pr->s_tol, f = 1.0;
                if (ratio > 1.2 * target) f = pr->tau;
                else if (ratio < 0.8 * target) f = 1.0 / pr->tau;
                if (f != 1.0) {
                    prm.rho1 *= f; prm.rho2 *= f; prm.rho3 *= f; prm.rho4 *= f;
                    for (size_t e = 0; e < ne; ++e) S->lam[e] /= f;
                    for (size_t e = 0; e < nc; ++e) S->mu[e] /= f;
                    for (size_t e = 0; e < np_; ++e) { S->p[e] /= f; S->nu[e] /= f; }
                }
            }
        }
    }
    rep->rho[0] = prm.rho1; rep->rho[1] = prm.rho2; rep->rho[2] = prm.rho3; rep->rho[3] = prm.rho4;
    free(xp); free(zp); free(gx); free(sp); free(colsum); free(hp);
    return 0;
}

/* ---- The iteration split over workers that own columns k ----------------
 * Step (a) and steps (e), (f), (g) act on one column (j, k) at a time
 * (Sec. II: the (j, k) updates are independent); the coupling along k is
 * the per-(i, j) sum of g(x) - lambda that steps (b), (d) and (i) use, and x
 * at k = 0 that steps (c) and (h) use (App. A).  A worker that owns the
 * columns [k0, k0 + n_s) of every row runs phase A on them; the partial
 * records of all workers are combined (sums; x at k = 0 from its owner;
 * maxima of the column residual terms); every worker then runs phase B with
 * the combined record.  Steps (d) and (i) take 1'z = sum_k (g(x) - lambda)
 * + n t, the value the monolithic iteration sums from the new z (equal up to
 * rounding).  P is the worker's slice of the problem (n = n_s columns; c
 * whole); S holds the worker's columns of x, z, lambda, s, mu and every
 * h, p, nu, x_1. */

/* Phase A: step (a), g(x), steps (e) and (f) on the worker's columns, then
 * its record rec[2mq + 2]: [0, mq) sum over its columns of g(x) - lambda
 * per pair (i, j); [mq, 2mq) x at the global k = 0 when k0 = 0, else 0;
 * [2mq] the largest demand residual |s - sum_i x + y| of its columns;
 * [2mq + 1] the largest |s - s~ - sum_i (x - x~)| (xprev, sprev: x and s
 * before the iteration). */
void orc_shard_phase_a(const orc_problem *P, const orc_params *pr, orc_state *S, int k0, const double *xprev,
                       const double *sprev, double *gx, double *colsum, double *rec)
{
    int n = P->n, m = P->m, q = P->q;
    orc_report scratch;
    memset(&scratch, 0, sizeof scratch);
    step_a(P, pr, S, xprev, k0, &scratch);
    for (size_t e = 0; e < (size_t)m * q * n; ++e)
        gx[e] = g_at(P, e, S->x[e]);
    steps_e_f(P, S, colsum);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double sum = 0.0;
            for (int k = 0; k < n; ++k)
                sum += gx[IDX3(i, j, k)] - S->lam[IDX3(i, j, k)];
            rec[(size_t)i * q + j] = sum;
            rec[(size_t)m * q + (size_t)i * q + j] = k0 == 0 ? S->x[IDX3(i, j, 0)] : 0.0;
        }
    double r1 = 0.0, s3 = 0.0;
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k) {
            double sx = 0.0, dx = 0.0;
            for (int i = 0; i < m; ++i) {
                sx += S->x[IDX3(i, j, k)];
                dx += S->x[IDX3(i, j, k)] - xprev[IDX3(i, j, k)];
            }
            r1 = amax(r1, fabs(S->s[IDX2(j, k)] - sx + P->y[IDX2(j, k)]));
            s3 = amax(s3, fabs(S->s[IDX2(j, k)] - sprev[IDX2(j, k)] - dx));
        }
    rec[2 * (size_t)m * q] = r1;
    rec[2 * (size_t)m * q + 1] = s3;
}

/* Phase B: with the combined record `tot`, step (b) on the worker's columns,
 * steps (c), (d), (h), (i) on the pair scalars (the same on every worker)
 * and step (g) on its columns; n_total is the instance's n.  res[0], res[1]
 * receive the worker's largest |z - g(x)| and |z - z~| (zprev: z before the
 * iteration); res[2..4] the largest |h - 1'z|, |x_1^(i,j) - x_1^(i)| and
 * |h - h~| over the pairs (hprev: h before), the same on every worker. */
void orc_shard_phase_b(const orc_problem *P, const orc_params *pr, orc_state *S, int n_total, const double *tot,
                       const double *gx, const double *zprev, const double *hprev, double *res)
{
    int n = P->n, m = P->m, q = P->q;
    size_t mq = (size_t)m * q;
    double kappa = pr->rho2 / (pr->rho1 + (double)n_total * pr->rho2);
    double r2 = 0.0, s1 = 0.0, r3 = 0.0, r4 = 0.0, s2 = 0.0;
    double *sz = malloc(sizeof(double) * mq);
    /* (b) z = g(x) - lambda + kappa (h + p - 1'(g(x) - lambda)) 1 */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            size_t pr_ = (size_t)i * q + j;
            double t = kappa * (S->h[pr_] + S->p[pr_] - tot[pr_]);
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                S->z[e] = gx[e] - S->lam[e] + t;
            }
            sz[pr_] = tot[pr_] + (double)n_total * t;
        }
    /* (c) x_1-update (R1) */
    for (int i = 0; i < m; ++i) {
        double sum = 0.0;
        for (int j = 0; j < q; ++j)
            sum += tot[mq + (size_t)i * q + j] - S->nu[(size_t)i * q + j];
        S->x1[i] = sum / (double)q;
    }
    /* (d) h-update */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            size_t pr_ = (size_t)i * q + j;
            double v = sz[pr_] - S->p[pr_];
            S->h[pr_] = v < P->c[i] ? v : P->c[i];
        }
    /* (g) lambda-update on the worker's columns, with the residual terms of z */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                r2 = amax(r2, fabs(S->z[e] - gx[e]));
                s1 = amax(s1, fabs(S->z[e] - zprev[e]));
                S->lam[e] += S->z[e] - gx[e];
            }
    /* (h) nu-update, (i) p-update, and the pair residual terms */
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            size_t pr_ = (size_t)i * q + j;
            double x0 = tot[mq + pr_];
            S->nu[pr_] += S->x1[i] - x0;
            S->p[pr_] += S->h[pr_] - sz[pr_];
            r3 = amax(r3, fabs(S->h[pr_] - sz[pr_]));
            r4 = amax(r4, fabs(x0 - S->x1[i]));
            s2 = amax(s2, fabs(S->h[pr_] - hprev[pr_]));
        }
    free(sz);
    res[0] = r2; res[1] = s1; res[2] = r3; res[3] = r4; res[4] = s2;
}

/* Objective of eq. (2): (1/q) sum_{i,j,k} f_k^{(i,j)}(x_k^{(i,j)}). */
double orc_objective(const orc_problem *P, const double *x)
{
    int n = P->n, m = P->m, q = P->q;
    double tot = 0.0;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j)
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                tot += P->f2[e] * x[e] * x[e] + P->f1[e] * x[e] + P->f0[e];
            }
    return tot / (double)q;
}

/* KKT residual of eq. (2) at x with multipliers recovered from the scaled
 * duals: eta = rho3 mu (demand), gamma = -rho2 p (capacity), omega = -rho4 nu
 * (copies x_1^{(i,j)} = x_1^{(i)}).  terms[]:
 *   0 projected-gradient stationarity  max |x - Pi(x - grad)|
 *   1 demand infeasibility             max (y - sum_i x)_+
 *   2 capacity infeasibility           max (sum_k g - c)_+
 *   3 copy infeasibility               max |x_1^{(i,j)} - x_1^{(i)}|
 *   4 demand complementarity           max |eta (sum_i x - y)|
 *   5 capacity complementarity         max |gamma (c - sum_k g)|  (0 if c = inf)
 *   6 dual sign                        max (-eta)_+, (-gamma)_+
 *   7 x_1 stationarity                 max_i |sum_j omega^{(i,j)}|
 * Returns the max of the terms. */
double orc_kkt(const orc_problem *P, const orc_params *pr, const orc_state *S, double *terms)
{
    int n = P->n, m = P->m, q = P->q;
    double t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) {
            double gamma = -pr->rho2 * S->p[(size_t)i * q + j];
            double omega = -pr->rho4 * S->nu[(size_t)i * q + j];
            double gsum = 0.0;
            for (int k = 0; k < n; ++k) {
                size_t e = IDX3(i, j, k);
                double x = S->x[e];
                double eta = pr->rho3 * S->mu[IDX2(j, k)];
                double grad = (2.0 * P->f2[e] * x + P->f1[e]) / (double)q
                              + gamma * (2.0 * P->g2[e] * x + P->g1[e]) - eta
                              + (k == 0 ? omega : 0.0);
                double pg = x - clampd(x - grad, P->lo[IDX2(i, k)], P->hi[IDX2(i, k)]);
                t[0] = amax(t[0], fabs(pg));
                gsum += g_at(P, e, x);
            }
            t[2] = amax(t[2], gsum - P->c[i]);
            if (isfinite(P->c[i]))
                t[5] = amax(t[5], fabs(gamma * (P->c[i] - gsum)));
            t[3] = amax(t[3], fabs(S->x[IDX3(i, j, 0)] - S->x1[i]));
            t[6] = amax(t[6], -gamma);
        }
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < n; ++k) {
            double sx = 0.0;
            for (int i = 0; i < m; ++i)
                sx += S->x[IDX3(i, j, k)];
            double eta = pr->rho3 * S->mu[IDX2(j, k)];
            t[1] = amax(t[1], P->y[IDX2(j, k)] - sx);
            t[4] = amax(t[4], fabs(eta * (sx - P->y[IDX2(j, k)])));
            t[6] = amax(t[6], -eta);
        }
    for (int i = 0; i < m; ++i) {
        double so = 0.0;
        for (int j = 0; j < q; ++j)
            so += -pr->rho4 * S->nu[(size_t)i * q + j];
        t[7] = amax(t[7], fabs(so));
    }
    double mx = 0.0;
    for (int a = 0; a < 8; ++a) {
        if (terms) terms[a] = t[a];
        mx = amax(mx, t[a]);
    }
    return mx;
}

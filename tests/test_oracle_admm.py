"""Pins of the oracle's ADMM iteration (App. A, (a)-(i)) and of its converged
solutions against definitions of L, invariants, closed forms, brute force and
an independent interior-point solve of eq. (2).  CPU only."""
import itertools
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from paper_1903_10041_gb300 import workloads as W
from tests._independent import barrier_solve, quartic_argmin_grid, waterfill_linear_capacity


def _random_state(prob, seed):
    """A non-zero iterate with lambda varying over k (so that the identities
    checked below are not trivially true)."""
    rng = np.random.default_rng(seed)
    m, q, n = prob.m, prob.q, prob.n
    x = np.clip(rng.uniform(-1, 2, (m, q, n)), prob.lo[:, None, :], prob.hi[:, None, :])
    return {"x": x, "z": rng.uniform(-1, 2, (m, q, n)), "lam": rng.uniform(-0.5, 0.5, (m, q, n)),
            "s": rng.uniform(0, 1, (q, n)), "mu": rng.uniform(0, 0.5, (q, n)),
            "h": rng.uniform(0, 5, (m, q)), "p": rng.uniform(-1, 0, (m, q)),
            "nu": rng.uniform(-0.3, 0.3, (m, q)), "x1": rng.uniform(0, 1, m)}


def _one_step(oracle, prob, st, **kw):
    par = W.Params(max_iter=1, r_tol=0.0, s_tol=0.0, **kw)
    return oracle.solve(prob, par, state=st)


def _g(prob, x):
    return prob.g2 * x * x + prob.g1 * x + prob.g0


@pytest.fixture
def small():
    return W.random_problem(7, 3, 4, seed=5)


def test_z_update_solves_its_linear_system(oracle_lib, small):
    """(b) minimises rho1/2 ||z - g + lambda||^2 + rho2/2 (h - 1'z + p)^2, i.e.
    (rho1 I + rho2 11') z = rho1 (g - lambda) + rho2 (h + p) 1."""
    rho = (0.7, 0.3, 1.1, 0.9)
    st0 = _random_state(small, 0)
    st1, _ = _one_step(oracle_lib, small, st0, rho=rho)
    g = _g(small, st1["x"])
    n = small.n
    M = rho[0] * np.eye(n) + rho[1] * np.ones((n, n))
    for i in range(small.m):
        for j in range(small.q):
            rhs = rho[0] * (g[i, j] - st0["lam"][i, j]) + rho[1] * (st0["h"][i, j] + st0["p"][i, j])
            z = np.linalg.solve(M, rhs)
            assert np.allclose(st1["z"][i, j], z, rtol=0, atol=1e-13)


def test_lambda_is_constant_over_k_after_one_iteration(oracle_lib, small):
    """(b) then (g): lambda_new = z - g + lambda_old is the same for every k."""
    st1, _ = _one_step(oracle_lib, small, _random_state(small, 1))
    lam = st1["lam"]
    assert np.abs(lam - lam[:, :, :1]).max() < 1e-13
    assert np.abs(lam).max() > 1e-3


@pytest.mark.parametrize("sweep", ["gauss_seidel", "jacobi"])
def test_x_update_minimises_L_over_each_element(oracle_lib, small, sweep):
    """(a): each x_k^(i,j) is the constrained minimiser of the x-terms of L,
    written from L's definition (not from the theta/phi form), with the
    other sources at their newest (Gauss-Seidel) or previous (Jacobi) values."""
    rho = (0.8, 0.5, 1.3, 0.6)
    st0 = _random_state(small, 2)
    st1, _ = _one_step(oracle_lib, small, st0, rho=rho, sweep=sweep)
    P, q = small, small.q
    for i, j, k in itertools.product(range(P.m), range(q), range(P.n)):
        others = sum((st1 if (sweep == "gauss_seidel" and l < i) else st0)["x"][l, j, k]
                     for l in range(P.m) if l != i)

        def Lx(x):
            gx = P.g2[i, j, k] * x * x + P.g1[i, j, k] * x + P.g0[i, j, k]
            v = (P.f2[i, j, k] * x * x + P.f1[i, j, k] * x) / q
            v += rho[0] / 2 * (st0["z"][i, j, k] - gx + st0["lam"][i, j, k]) ** 2
            v += rho[2] / 2 * (st0["s"][j, k] - (x + others) + P.y[j, k] + st0["mu"][j, k]) ** 2
            if k == 0:
                v += rho[3] / 2 * (st0["x1"][i] - x + st0["nu"][i, j]) ** 2
            return v

        # expand Lx into a quartic by exact polynomial fitting (5 points)
        pts = np.array([-2.0, -1.0, 0.0, 1.0, 2.0])
        cf = np.polyfit(pts, [Lx(t) for t in pts], 4)  # A B C D E
        xb, fb, gap = quartic_argmin_grid(cf[0], cf[1], cf[2], cf[3], P.lo[i, k], P.hi[i, k])
        x = st1["x"][i, j, k]
        assert Lx(x) <= Lx(xb) + 1e-11 * max(1, abs(Lx(xb)))
        if gap > 1e-8:
            assert abs(x - xb) < 1e-7


def test_x1_h_s_updates_minimise_their_terms_of_L(oracle_lib, small):
    """(c), (d), (e) minimise L over x_1, h <= c and s >= 0; checked by scalar
    numerical minimisation of the terms of L."""
    rho = (0.9, 0.4, 1.2, 0.7)
    st0 = _random_state(small, 3)
    st1, _ = _one_step(oracle_lib, small, st0, rho=rho)
    P = small
    x, z = st1["x"], st1["z"]
    for i in range(P.m):
        f = lambda v: sum((v - x[i, j, 0] + st0["nu"][i, j]) ** 2 for j in range(P.q))
        res = minimize_scalar(f, bracket=(-10, 10), tol=1e-12)
        assert abs(st1["x1"][i] - res.x) < 1e-7
        for j in range(P.q):
            hz = z[i, j].sum()
            f = lambda v: (v - hz + st0["p"][i, j]) ** 2
            res = minimize_scalar(f, bounds=(hz - 1e3, P.c[i]), method="bounded",
                                  options={"xatol": 1e-12})
            assert abs(st1["h"][i, j] - res.x) < 1e-6
            assert st1["h"][i, j] <= P.c[i]
    sx = x.sum(axis=0)
    for j, k in itertools.product(range(P.q), range(P.n)):
        f = lambda v: (v - sx[j, k] + P.y[j, k] + st0["mu"][j, k]) ** 2
        res = minimize_scalar(f, bounds=(0.0, 100.0), method="bounded", options={"xatol": 1e-12})
        assert abs(st1["s"][j, k] - res.x) < 1e-6


def test_invariants_hold_along_a_run(oracle_lib):
    """After every iteration: mu >= 0 and s * mu = 0 ((e)+(f)); p <= 0 ((d)+(i));
    sum_j nu = 0 ((c)+(h)); lambda constant over k ((b)+(g))."""
    P = W.random_problem(20, 2, 3, seed=6)
    par = W.Params(max_iter=1, r_tol=0.0, s_tol=0.0)
    st, _ = oracle_lib.solve(P, par)
    for _ in range(40):
        st, _ = oracle_lib.solve(P, par, state=st)
        # (f) is applied literally, so the identities hold up to one rounding
        assert st["mu"].min() >= -1e-15
        assert np.abs(st["s"] * st["mu"]).max() <= 1e-14
        assert st["p"].max() <= 1e-15
        assert np.abs(st["nu"].sum(axis=1)).max() < 1e-13
        assert np.abs(st["lam"] - st["lam"][:, :, :1]).max() < 1e-12


def test_primal_residual_bounds_infeasibility_of_eq2(oracle_lib):
    """r bounds the violations of eq. (2): demand <= r, copies <= r and
    capacity <= (n + 1) r (s >= 0, z = g + O(r), h <= c)."""
    P = W.random_problem(15, 3, 2, seed=7)
    par = W.Params(max_iter=1, r_tol=0.0, s_tol=0.0, check_every=1)
    st = None
    for _ in range(60):
        st, rep = oracle_lib.solve(P, par, state=st)
        r = rep["r"]
        x = st["x"]
        dem = (P.y - x.sum(axis=0)).max()
        cap = (_g(P, x).sum(axis=2) - P.c[:, None]).max()
        cop = np.abs(x[:, :, 0] - st["x1"][:, None]).max()
        assert dem <= r * (1 + 1e-12) + 1e-15
        assert cop <= r * (1 + 1e-12) + 1e-15
        assert cap <= (P.n + 1) * r * (1 + 1e-12) + 1e-12


def test_residuals_vanish_at_a_fixed_point(oracle_lib):
    P = W.random_problem(10, 2, 2, seed=8)
    par = W.Params(r_tol=1e-13, s_tol=1e-13, max_iter=200000)
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    st2, rep2 = oracle_lib.solve(P, par.replace(max_iter=1, r_tol=0, s_tol=0), state=st)
    assert rep2["r"] < 1e-12 and rep2["sigma"] < 1e-12


@pytest.mark.parametrize("n,m,q", [(100, 2, 1), (30, 3, 3), (25, 2, 5)])
def test_converged_solution_satisfies_kkt(oracle_lib, n, m, q):
    P = W.random_problem(n, m, q, seed=9 + n)
    par = W.Params(rho=(1.0, 1.0 / n, 1.0, 1.0))
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    k, terms = oracle_lib.kkt(P, par, st)
    assert k < 5e-6, terms


@pytest.mark.parametrize("n,m,q,seed", [(6, 2, 1, 10), (5, 3, 2, 11), (4, 2, 3, 12)])
def test_converged_solution_matches_interior_point(oracle_lib, n, m, q, seed):
    """Strictly convex objective (f2 > 0): x* is unique; the oracle at tight
    tolerance equals a log-barrier interior-point solution of eq. (2)."""
    P = W.random_problem(n, m, q, seed=seed)
    # sources want to run high; capacities just above the barrier's start
    # point (x = y/m + 0.05) keep eq. (2) strictly feasible and make them bind
    P.f1[:] = -np.abs(P.f1) - 0.5
    x0 = np.broadcast_to(P.y[None] / m + 0.05, (m, q, n)).copy()
    x0[:, :, 0] = P.y[:, 0].max() / m + 0.05
    P.c = 1.02 * _g(P, x0).sum(axis=2).max(axis=1)
    par = W.Params(r_tol=1e-11, s_tol=1e-11, max_iter=400000, check_every=10)
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    assert (-st["p"]).max() > 1e-6  # a capacity multiplier is active
    xb = barrier_solve(P)
    assert np.abs(st["x"] - xb).max() < 1e-6
    assert abs(oracle_lib.objective(P, st["x"]) - oracle_lib.objective(P, xb)) < 1e-8


def test_converged_objective_matches_brute_force_grid(oracle_lib):
    """n = 2, m = 2, q = 1: the oracle's optimum against a 4-D grid over the
    box (step h): obj <= grid best + 1e-9 and >= grid best - L h."""
    P = W.random_problem(2, 2, 1, seed=13)
    P.f1[:] = -np.abs(P.f1) - 0.5
    P.c = 1.1 * _g(P, np.broadcast_to(P.y[None] / 2 + 0.05, (2, 1, 2))).sum(axis=2).max(axis=1)
    par = W.Params(r_tol=1e-11, s_tol=1e-11, max_iter=400000)
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    assert (-st["p"]).max() > 1e-6  # a capacity multiplier is active
    N = 61
    ax = np.linspace(-1.0, 2.0, N)
    h = ax[1] - ax[0]
    X = np.stack(np.meshgrid(ax, ax, ax, ax, indexing="ij"), -1).reshape(-1, 2, 1, 2)  # [pt, i, j, k]
    obj = (P.f2[None] * X * X + P.f1[None] * X).sum(axis=(1, 2, 3))
    dem = X.sum(axis=1)[:, 0, :] >= P.y[0][None, :]
    cap = ((P.g2[None] * X * X + P.g1[None] * X).sum(axis=3)[:, :, 0] <= P.c[None, :]).all(axis=1)
    ok = dem.all(axis=1) & cap
    best = obj[ok].min()
    o = oracle_lib.objective(P, st["x"])
    lip = np.abs(2 * P.f2 * 2.0 + P.f1).sum()
    assert o <= best + 1e-9
    assert o >= best - lip * h


def test_closed_form_unconstrained_when_demand_slack_and_no_capacity(oracle_lib):
    P = W.random_problem(30, 2, 2, seed=14)
    P.y[:] = -10.0
    P.c[:] = np.inf
    st, rep = oracle_lib.solve(P, W.Params(r_tol=1e-10, s_tol=1e-10, max_iter=100000))
    assert rep["converged"]
    want = np.clip(-P.f1 / (2 * P.f2), -1.0, 2.0)
    # x_1 copies: the shared first move averages nothing away when each
    # scenario's minimiser differs, so compare k >= 1 exactly and k = 0 by KKT
    assert np.abs(st["x"][:, :, 1:] - want[:, :, 1:]).max() < 1e-7


def test_closed_form_single_source_meets_demand(oracle_lib):
    P = W.random_problem(40, 1, 1, seed=15)
    P.c[:] = np.inf
    st, rep = oracle_lib.solve(P, W.Params(r_tol=1e-10, s_tol=1e-10, max_iter=100000))
    assert rep["converged"]
    want = np.clip(np.maximum(-P.f1[0, 0] / (2 * P.f2[0, 0]), P.y[0]), -1.0, 2.0)
    assert np.abs(st["x"][0, 0] - want).max() < 1e-7


def test_closed_form_water_filling_with_linear_losses(oracle_lib):
    """beta_2 = 0, demand slack, binding capacity: x_k(gamma) with gamma by bisection."""
    P = W.random_problem(50, 1, 1, seed=16)
    P.g2[:] = 0.0
    P.g1[:] = np.random.default_rng(16).uniform(0.5, 1.5, P.g1.shape)
    P.f1[:] = -np.abs(P.f1) - 0.5  # every source wants to run high
    P.y[:] = -10.0
    P.c[:] = 10.0
    st, rep = oracle_lib.solve(P, W.Params(r_tol=1e-10, s_tol=1e-10, max_iter=200000))
    assert rep["converged"]
    want, gamma = waterfill_linear_capacity(P.f2[0, 0], P.f1[0, 0], P.g1[0, 0], -1.0, 2.0, 10.0, 1)
    assert gamma > 0
    assert np.abs(st["x"][0, 0] - want).max() < 1e-7


def test_adaptive_rho_reaches_the_same_solution(oracle_lib):
    """Sec. IV-A penalty adaptation with dual rescaling changes the path, not x*."""
    P = W.random_problem(60, 2, 3, seed=17)
    par = W.Params(rho=(1.0, 1.0 / 60, 1.0, 1.0), r_tol=1e-9, s_tol=1e-9, max_iter=200000)
    st0, rep0 = oracle_lib.solve(P, par)
    st1, rep1 = oracle_lib.solve(P, par.replace(adapt_rho=True))
    assert rep0["converged"] and rep1["converged"]
    assert rep1["rho"][0] != 1.0
    assert np.abs(st0["x"] - st1["x"]).max() < 1e-6
    k, terms = oracle_lib.kkt(P, par.replace(rho=tuple(rep1["rho"])), st1)
    assert k < 1e-7, terms


def test_late_adaptation_is_fixed_rho_then_adaptive_continuation(oracle_lib):
    """adapt_start = T0 + 1 (T0 a check iteration): T0 iterations at fixed
    rho (a solve with max_iter = T0 never adapts at its last iteration), then
    the adaptive iteration resumed from that state, give the same iterates,
    penalties and iteration count as one solve.  adapt_start beyond the last
    check is the fixed-rho solve; adapt_start = 0 the adaptive one."""
    P = W.random_problem(50, 2, 3, seed=19)
    par = W.Params(rho=(1.0, 1.0 / 50, 1.0, 1.0), r_tol=1e-8, s_tol=1e-8, max_iter=3000, adapt_rho=True)
    T0 = 120
    st, rep = oracle_lib.solve(P, par.replace(adapt_start=T0 + 1))
    s1, r1 = oracle_lib.solve(P, par.replace(adapt_rho=False, max_iter=T0))
    assert not r1["converged"]
    s2, r2 = oracle_lib.solve(P, par.replace(max_iter=par.max_iter - T0), state=s1)
    assert rep["converged"] and r2["converged"]
    assert rep["iters"] == T0 + r2["iters"] and rep["rho"] == r2["rho"] and rep["rho"][0] != 1.0
    for k in ("x", "z", "lam", "s", "mu", "h", "p", "nu", "x1"):
        assert np.array_equal(st[k], s2[k]), k
    sf, rf = oracle_lib.solve(P, par.replace(adapt_rho=False))
    sl, rl = oracle_lib.solve(P, par.replace(adapt_start=par.max_iter + 1))
    assert rl["iters"] == rf["iters"] and np.array_equal(sl["x"], sf["x"])
    sa, ra = oracle_lib.solve(P, par)
    s0, r0 = oracle_lib.solve(P, par.replace(adapt_start=0))
    assert r0["iters"] == ra["iters"] and np.array_equal(s0["x"], sa["x"])


def test_dual_residual_bounds_z_stationarity_violation(oracle_lib):
    """Stationarity of L in z asks rho1 lambda = rho2 p.  After (b), (g), (i)
    it is violated by exactly rho2 (h - h~), so sigma >= max |rho1 lambda -
    rho2 p| at every iterate, with equality while the h-term dominates."""
    P = W.random_problem(20, 2, 2, seed=18)
    P.f1[:] = -np.abs(P.f1) - 0.5
    P.c = 0.3 * P.c
    rho = (1.0, 0.7, 1.0, 1.0)
    par = W.Params(rho=rho, max_iter=1, r_tol=0.0, s_tol=0.0, check_every=1)
    st, equal = None, 0
    for _ in range(80):
        st, rep = oracle_lib.solve(P, par, state=st)
        viol = np.abs(rho[0] * st["lam"] - rho[1] * st["p"][:, :, None]).max()
        assert rep["sigma"] >= viol * (1 - 1e-9) - 1e-14
        equal += abs(rep["sigma"] - viol) <= 1e-9 * viol
    assert equal >= 1


def test_penalty_change_keeps_a_fixed_point(oracle_lib):
    """The scaled duals lambda, p, mu, nu carry a factor 1/rho, so the
    rescaling that goes with a Sec. IV-A penalty change (reading R11) keeps
    the unscaled multipliers, and with them a fixed point of the iteration:
    once converged, further iterations under repeated penalty changes leave x
    where it is.  A missing or inverted rescaling moves it by O(1)."""
    P = W.random_problem(60, 2, 3, seed=17)
    par = W.Params(rho=(1.0, 1.0 / 60, 1.0, 1.0), r_tol=1e-11, s_tol=1e-11, max_iter=200000)
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    # thresholds that are never met, so the ratio test changes rho at every check
    cont = par.replace(adapt_rho=True, r_tol=1e-30, s_tol=1e-30, check_every=1, max_iter=40)
    st2, rep2 = oracle_lib.solve(P, cont, state=st)
    assert abs(math.log(rep2["rho"][0])) > 5 * math.log(1.1)  # several changes took place
    assert np.abs(st2["x"] - st["x"]).max() < 1e-8
    assert rep2["r"] < 1e-10 and rep2["sigma"] < 1e-10


def test_kkt_residual_reports_each_kind_of_violation(oracle_lib):
    """The KKT residual is the bar the mixed-precision results are held to,
    so each of its terms must respond to the violation it measures: starting
    from a converged iterate, break one condition of eq. (2) or one dual
    condition at a time and check that its term (and the max) rises."""
    P = W.random_problem(25, 2, 5, seed=34)
    par = W.Params(rho=(1.0, 1.0 / 25, 1.0, 1.0), r_tol=1e-9, s_tol=1e-9, max_iter=200000)
    st, rep = oracle_lib.solve(P, par)
    assert rep["converged"]
    k0, t0 = oracle_lib.kkt(P, par, st)
    assert k0 < 1e-7, t0
    sx = st["x"].sum(axis=0)                               # [q, n]
    gsum = (P.g2 * st["x"] ** 2 + P.g1 * st["x"] + P.g0).sum(axis=2)  # [m, q]

    def term(t, st2=None, P2=None):
        k, tt = oracle_lib.kkt(P2 or P, par, st2 or st)
        assert k >= tt[t] and k == tt.max()
        return tt[t]

    def edit(**arrs):
        s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
        for k, f in arrs.items():
            f(s2[k])
        return s2

    lo, hi = P.lo[:, None, :], P.hi[:, None, :]
    i, j, k = np.argwhere((st["x"] > lo + 0.05) & (st["x"] < hi - 0.05) &
                          (np.arange(P.n)[None, None, :] > 0))[0]
    assert term(0, edit(x=lambda a: a.__setitem__((i, j, k), a[i, j, k] + 0.02))) > 1e-4   # stationarity
    jb, kb = np.argwhere(st["mu"] > 1e-3)[0]                # a binding demand (eta > 0)
    assert term(1, edit(x=lambda a: a.__setitem__((slice(None), jb, kb), a[:, jb, kb] - 0.05))) > 0.05
    P2 = P.copy()
    P2.c = 0.5 * gsum.min(axis=1)
    assert term(2, P2=P2) > 0.1                             # capacity infeasible
    assert term(3, edit(x=lambda a: a.__setitem__((0, 1, 0), a[0, 1, 0] + 0.1))) > 0.09     # copies differ
    js, ks = np.argwhere(sx - P.y > 0.05)[0]                # a slack demand
    assert term(4, edit(mu=lambda a: a.__setitem__((js, ks), 1.0))) > 0.04                 # eta (sum x - y) != 0
    ic, jc = np.argwhere(gsum < P.c[:, None] - 0.05)[0]     # a slack capacity
    assert term(5, edit(p=lambda a: a.__setitem__((ic, jc), -25.0))) > 0.04               # gamma (c - sum g) != 0
    assert term(6, edit(mu=lambda a: a.__setitem__((0, 0), -0.5))) >= 0.5                  # eta < 0
    assert term(7, edit(nu=lambda a: a.__setitem__((0, 0), a[0, 0] + 0.5))) >= 0.5 - 1e-12  # sum_j omega != 0


def test_residual_terms_equal_the_dual_increments(oracle_lib, small):
    """In scaled form each dual step adds the residual of its constraint
    (steps (f)-(i)), so the primal residual terms of App. A are the largest
    dual increments of the same iteration: demand |s - sum x + y| = |d mu|,
    losses |z - g(x)| = |d lambda|, capacity copies |h - 1'z| = |d p|, x_1
    copies |x_1^(i,j) - x_1^(i)| = |d nu|; and the demand dual-residual term
    rho3 |d s - sum d x| = rho3 |d mu - d mu_prev| (the change between two
    consecutive increments of mu, since y is fixed)."""
    rho = (1.3, 0.4, 0.7, 1.1)
    par = W.Params(rho=rho, max_iter=1, r_tol=0.0, s_tol=0.0, check_every=1)
    P = small.copy()
    P.c = 0.3 * P.c  # binding capacities, so that h is clipped and p moves
    st0 = _random_state(P, 77)
    st1, _ = oracle_lib.solve(P, par, state=st0)
    st2, rep = oracle_lib.solve(P, par, state=st1)
    r_mu, r_lam, r_p, r_nu = rep["r_terms"]
    d = {k: st2[k] - st1[k] for k in ("mu", "lam", "p", "nu")}
    assert r_mu == pytest.approx(np.abs(d["mu"]).max(), rel=1e-12, abs=1e-14)
    assert r_lam == pytest.approx(np.abs(d["lam"]).max(), rel=1e-12, abs=1e-14)
    assert r_p == pytest.approx(np.abs(d["p"]).max(), rel=1e-12, abs=1e-14)
    assert r_nu == pytest.approx(np.abs(d["nu"]).max(), rel=1e-12, abs=1e-14)
    assert min(r_mu, r_lam, r_p, r_nu) > 1e-6  # a non-trivial iterate
    second = (st2["mu"] - st1["mu"]) - (st1["mu"] - st0["mu"])
    assert rep["s_terms"][2] == pytest.approx(rho[2] * np.abs(second).max(), rel=1e-12, abs=1e-14)
    assert rep["s_terms"][2] > 1e-6


@pytest.mark.parametrize("band", ["grow", "hold", "shrink"])
def test_penalty_adaptation_follows_the_ratio_rule(oracle_lib, band):
    """Sec. IV-A: every rho_t grows by tau when r / sigma > 1.2 rbar/sbar,
    shrinks by tau when r / sigma < 0.8 rbar/sbar, and stays in between.  The
    first check (after 10 iterations) decides the penalties used from
    iteration 11 on; thresholds far below reach are chosen so that no stop
    intervenes, with rbar/sbar placed relative to the observed ratio."""
    P = W.random_problem(30, 2, 3, seed=21)
    rho0 = (1.0, 1.0 / 30, 1.0, 1.0)
    base = W.Params(rho=rho0, r_tol=1e-30, s_tol=1e-30, check_every=10, adapt_rho=True, tau=1.1)
    _, rep10 = oracle_lib.solve(P, base.replace(max_iter=10))  # the last iteration never adapts
    assert rep10["rho"] == list(rho0)
    ratio = rep10["r"] / rep10["sigma"]
    target, f = {"grow": (ratio / 1.5, 1.1), "hold": (ratio, 1.0), "shrink": (ratio / 0.6, 1.0 / 1.1)}[band]
    _, rep20 = oracle_lib.solve(P, base.replace(max_iter=20, r_tol=target * 1e-30))
    assert rep20["rho"] == pytest.approx([f * r for r in rho0], rel=1e-15)


def test_objective_invariances(oracle_lib):
    """The objective of eq. (2) is the scenario mean of the nominal cost (1):
    q identical scenarios give the nominal value; shifting every f0 by d
    shifts it by n m d; it is linear in (f2, f1, f0) jointly."""
    rng = np.random.default_rng(5)
    P1 = W.random_problem(40, 3, 1, seed=61)
    x1 = rng.uniform(P1.lo[:, None, :], P1.hi[:, None, :], (3, 1, 40))
    q = 7
    Pq = P1.copy()
    for k in ("f2", "f1", "f0", "g2", "g1", "g0"):
        setattr(Pq, k, np.repeat(getattr(P1, k), q, axis=1))
    Pq.y = np.repeat(P1.y, q, axis=0)
    Pq.q = q
    xq = np.repeat(x1, q, axis=1)
    v1 = oracle_lib.objective(P1, x1)
    assert oracle_lib.objective(Pq, xq) == pytest.approx(v1, rel=1e-13)
    Ps = Pq.copy()
    Ps.f0 = Pq.f0 + 0.25
    assert oracle_lib.objective(Ps, xq) - oracle_lib.objective(Pq, xq) == pytest.approx(40 * 3 * 0.25, rel=1e-12)
    P2 = Pq.copy()
    P2.f2, P2.f1, P2.f0 = 2 * Pq.f2, 2 * Pq.f1, 2 * Pq.f0
    assert oracle_lib.objective(P2, xq) == pytest.approx(2 * oracle_lib.objective(Pq, xq), rel=1e-13)
    assert abs(v1) > 1.0  # non-trivial value
    # a quadratic in every element: the second difference along a uniform
    # shift h is 2 h^2 sum(f2) / q, whatever the point
    h = 0.5
    d2 = (oracle_lib.objective(Pq, xq + h) - 2 * oracle_lib.objective(Pq, xq) +
          oracle_lib.objective(Pq, xq - h))
    assert d2 == pytest.approx(2 * h * h * Pq.f2.sum() / q, rel=1e-10)


def test_open_loop_variant_is_the_nominal_problem_on_the_largest_demand(oracle_lib):
    """Sec. II's open-loop formulation (one sequence per source against
    max_j y_k^(j)) is problem (1) with that demand, so it is solved as q = 1.
    Repeated over the scenarios, its solution is feasible for eq. (2) (same
    first move, every scenario's demand met, same capacities), so the
    receding-horizon optimum of eq. (2) costs no more than it."""
    P = W.shared_problem(30, 2, 4, seed=71).dense()  # cost and loss maps shared by the scenarios
    par = W.Params(rho=(1.0, 1.0 / 30, 1.0, 1.0), r_tol=1e-9, s_tol=1e-9, max_iter=200000)
    st_r, rep_r = oracle_lib.solve(P, par)
    assert rep_r["converged"]
    ol = P.copy()
    for k in ("f2", "f1", "f0", "g2", "g1", "g0"):
        setattr(ol, k, np.ascontiguousarray(getattr(P, k)[:, :1, :]))
    ol.y = P.y.max(axis=0, keepdims=True)
    ol.q = 1
    st_o, rep_o = oracle_lib.solve(ol, par)
    assert rep_o["converged"]
    x_rep = np.repeat(st_o["x"], P.q, axis=1)
    assert (x_rep.sum(axis=0) >= P.y - 1e-6).all()                                   # demand of every scenario
    gsum = (P.g2 * x_rep ** 2 + P.g1 * x_rep + P.g0).sum(axis=2)
    assert (gsum <= P.c[:, None] + 1e-6).all()                                        # capacities
    obj_ol = oracle_lib.objective(P, x_rep)
    assert obj_ol == pytest.approx(oracle_lib.objective(ol, st_o["x"]), rel=1e-12)
    obj_r = oracle_lib.objective(P, st_r["x"])
    assert obj_r <= obj_ol + 1e-6
    assert obj_r < obj_ol - 1e-3  # scenario feedback after the first move pays on this instance


def test_start_point_does_not_change_the_solution(oracle_lib):
    """Reading R8 starts from x = Pi(0), the paper gives no start.  The start
    fixes the trajectory only: with f strictly convex (f2 > 0) eq. (2) has
    one minimiser, and solves from Pi(0), from x = 0 outside the bounds and
    from a random iterate reach it."""
    P = W.random_problem(60, 2, 3, seed=23)
    P.lo = np.full_like(P.lo, 0.25)       # 0 lies outside [lo, hi]: Pi(0) != 0
    par = W.Params(rho=(1.0, 1.0 / 60, 1.0, 1.0), r_tol=1e-9, s_tol=1e-9, max_iter=200000)
    st_a, rep_a = oracle_lib.solve(P, par)
    assert np.all(oracle_lib.init_state(P)["x"] == 0.25)
    zero = {k: np.zeros_like(v) for k, v in oracle_lib.init_state(P).items()}
    st_b, rep_b = oracle_lib.solve(P, par, state=zero)
    st_c, rep_c = oracle_lib.solve(P, par, state=_random_state(P, 29))
    assert rep_a["converged"] and rep_b["converged"] and rep_c["converged"]
    assert rep_a["iters"] != rep_b["iters"] or np.abs(st_a["x"] - st_b["x"]).max() > 0.0
    for st in (st_b, st_c):
        assert np.abs(st["x"] - st_a["x"]).max() < 1e-6
        assert abs(oracle_lib.objective(P, st["x"]) - oracle_lib.objective(P, st_a["x"])) < 1e-8

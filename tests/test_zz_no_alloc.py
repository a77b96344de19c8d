"""The allocation-free entry point admm_solve_noalloc, for callers that
cannot allocate device memory (host callbacks and real-time loops where an
allocation may block or fail, fixed-budget controllers, plugins whose host
application owns every allocation).  Its output must equal admm_solve's,
within the 1e-9 relative tolerance of the parity tests, on two calls in a
row: the second call reuses the fixed scratch array the first one left
behind.  Also: an odd, ragged n; a warm re-solve from the state a call left
behind; no device memory taken by a call after the first; invalid problems
rejected before the caller's state is written.  This file is collected last
so that a run stopping at the first failure has already run every other
test."""
import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9
STATE_KEYS = ("x", "s", "mu", "lam", "zeta", "h", "p", "nu", "x1")


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return torch, capi


def _device_problem(P, torch):
    D = P.copy()
    for k, v in P.arrays().items():
        setattr(D, k, torch.from_numpy(np.ascontiguousarray(v)).cuda())
    return D


def _zero_state(P, par, torch, fill=0.0):
    z = lambda *s: torch.full(s, fill, dtype=torch.float64, device="cuda")
    m, q, n = P.m, P.q, P.n
    return {"x": z(m, q, n), "s": z(q, n), "mu": z(q, n), "lam": z(m, q), "zeta": z(m, q), "h": z(m, q),
            "p": z(m, q), "nu": z(m, q), "x1": z(m), "rho": list(par.rho), "cold": True}


def _host_state(st):
    return {k: st[k].cpu().numpy() for k in STATE_KEYS}


def _check_equal(res, st, ref, st_ref):
    assert res["iters"] == ref["iters"] and res["converged"] == ref["converged"]
    assert abs(res["objective"] - ref["objective"]) <= TOL * max(1.0, abs(ref["objective"]))
    for k in STATE_KEYS:
        assert rel(st[k].cpu().numpy(), st_ref[k]) <= TOL, k


CASES = [
    (lambda: W.config(0), W.Params()),                                                # to convergence
    (lambda: W.random_problem(300, 3, 4, seed=71),
     W.Params(rho=(1.0, 1.0 / 300, 1.0, 1.0), max_iter=200, r_tol=0.0, s_tol=0.0)),
    (lambda: W.random_problem(4099, 2, 3, seed=73),                                   # odd n: rows not 32-aligned
     W.Params(rho=(1.0, 1.0 / 4099, 1.0, 1.0), max_iter=120, r_tol=0.0, s_tol=0.0)),
]


def test_noalloc_matches_admm_solve_on_two_calls_in_a_row(env):
    torch, capi = env
    for mk, par in CASES:
        P = mk()
        D = _device_problem(P, torch)
        st = _zero_state(P, par, torch)
        res = capi.admm_solve_noalloc(D, par, st)
        with capi.Solver(P, par) as s:
            ref = s.solve(raise_on=(1, 2, 3, 4, 6))
            st_ref = s.state()
        _check_equal(res, st, ref, st_ref)
        assert st["cold"] is False and st_ref["cold"] is False


def test_noalloc_warm_resolve_after_a_data_change(env):
    """A re-solve from the state the previous call left behind (cold = 0),
    as a receding-horizon controller makes it: the demand moves one step
    forward and the solve continues from the old duals."""
    torch, capi = env
    P = W.random_problem(500, 2, 3, seed=77)
    par = W.Params(rho=(1.0, 1.0 / 500, 1.0, 1.0))
    D = _device_problem(P, torch)
    st = _zero_state(P, par, torch)
    capi.admm_solve_noalloc(D, par, st)
    with capi.Solver(P, par) as s:
        s.solve(raise_on=(1, 2, 3, 4, 6))
        st_ref = s.state()
    P2 = P.copy()
    P2.y = np.ascontiguousarray(np.concatenate([P.y[:, 1:], P.y[:, -1:]], axis=1))
    D2 = _device_problem(P2, torch)
    res = capi.admm_solve_noalloc(D2, par, st)
    with capi.Solver(P2, par) as s:
        ref = s.solve(warm=st_ref, raise_on=(1, 2, 3, 4, 6))
        st_ref2 = s.state()
    assert 0 < ref["iters"] < 5000
    _check_equal(res, st, ref, st_ref2)


def test_noalloc_takes_no_device_memory_after_the_first_call(env):
    torch, capi = env
    P, par = CASES[1][0](), CASES[1][1]
    D = _device_problem(P, torch)
    st = _zero_state(P, par, torch)
    capi.admm_solve_noalloc(D, par, st)            # warm-up: module load and symbol look-up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    st["cold"] = True
    capi.admm_solve_noalloc(D, par, st)
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert alloc1 == alloc0
    assert free1 == free0, (free0, free1)


@pytest.mark.parametrize("bad", ["nan_coefficient", "lo_above_hi", "infeasible_capacity"])
def test_noalloc_rejects_invalid_data_before_writing_the_state(env, bad):
    torch, capi = env
    P = W.random_problem(97, 2, 3, seed=79)
    par = W.Params(rho=(1.0, 1.0 / 97, 1.0, 1.0))
    if bad == "nan_coefficient":
        P.f1[1, 2, 50] = np.nan
    elif bad == "lo_above_hi":
        P.lo[0, 10], P.hi[0, 10] = 1.0, 0.5
    else:
        P.c[1] = -1e6  # far below sum_k min_{[lo, hi]} g (about -n)
    D = _device_problem(P, torch)
    st = _zero_state(P, par, torch, fill=7.0)      # a cold start would overwrite x, s, mu
    before = _host_state(st)
    with pytest.raises(capi.AdmmError) as e:
        capi.admm_solve_noalloc(D, par, st)
    assert e.value.status == capi.ADMM_EINVAL
    after = _host_state(st)
    for k in STATE_KEYS:
        assert np.array_equal(before[k], after[k]), k
    assert st["cold"] is True


def test_noalloc_rejects_shapes_beyond_the_limits(env):
    torch, capi = env
    P = W.random_problem(16, 9, 1, seed=81)        # m > ADMM_MAX_M
    par = W.Params()
    D = _device_problem(P, torch)
    st = _zero_state(P, par, torch)
    with pytest.raises(capi.AdmmError) as e:
        capi.admm_solve_noalloc(D, par, st)
    assert e.value.status == capi.ADMM_EUNSUPPORTED

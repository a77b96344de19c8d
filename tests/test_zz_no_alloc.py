"""The allocation-free entry point admm_solve_noalloc, for callers that
cannot allocate device memory (host callbacks and real-time loops where an
allocation may block or fail, fixed-budget controllers, plugins whose host
application owns every allocation).  Its output must equal admm_solve's,
within the 1e-9 relative tolerance of the parity tests, on two calls in a
row: the second call reuses the fixed scratch array the first one left
behind.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def _device_problem(P, torch):
    D = P.copy()
    for k, v in P.arrays().items():
        setattr(D, k, torch.from_numpy(np.ascontiguousarray(v)).cuda())
    return D


def _zero_state(P, par, torch):
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    m, q, n = P.m, P.q, P.n
    return {"x": z(m, q, n), "s": z(q, n), "mu": z(q, n), "lam": z(m, q), "zeta": z(m, q), "h": z(m, q),
            "p": z(m, q), "nu": z(m, q), "x1": z(m), "rho": list(par.rho), "cold": True}


def test_noalloc_matches_admm_solve_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi

    cases = [
        (W.config(0), W.Params()),                                           # to convergence
        (W.random_problem(300, 3, 4, seed=71),
         W.Params(rho=(1.0, 1.0 / 300, 1.0, 1.0), max_iter=200, r_tol=0.0, s_tol=0.0)),
    ]
    for P, par in cases:
        D = _device_problem(P, torch)
        st = _zero_state(P, par, torch)
        res = capi.admm_solve_noalloc(D, par, st)
        with capi.Solver(P, par) as s:
            ref = s.solve(raise_on=(1, 2, 3, 4, 6))
            st_ref = s.state()
        assert res["iters"] == ref["iters"] and res["converged"] == ref["converged"]
        assert abs(res["objective"] - ref["objective"]) <= TOL * max(1.0, abs(ref["objective"]))
        for k in ("x", "s", "mu", "lam", "zeta", "h", "p", "nu", "x1"):
            assert rel(st[k].cpu().numpy(), st_ref[k]) <= TOL, k
        assert st["cold"] is False and st_ref["cold"] is False

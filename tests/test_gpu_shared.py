"""Scenario-shared cost and loss maps (f and g drawn per (i, k), stored once
as [m][n]): single-instance, batched and served solves give the same bits
as on the same problem with the maps repeated for every scenario, and match
the oracle (which takes the repeated, dense form)."""
import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_maps_give_the_bits_of_the_dense_problem(capi, precision):
    P = W.shared_problem(777, 3, 6, seed=21)
    par = W.Params(rho=(1.0, 1.0 / 777, 1.0, 1.0), precision=precision)
    out = []
    for Q in (P, P.dense()):
        with capi.Solver(Q, par) as s:
            res = s.solve(raise_on=(1, 2, 3, 4, 6))
            out.append((res, s.state()))
    (r_s, st_s), (r_d, st_d) = out
    assert r_s["converged"] and r_s["iters"] == r_d["iters"]
    for k in ("x", "s", "mu", "lam", "h", "p", "nu", "x1"):
        assert np.array_equal(st_s[k], st_d[k]), k


def test_shared_maps_match_the_oracle(capi, oracle_lib):
    P = W.shared_problem(500, 2, 4, seed=22)
    par = W.Params(rho=(1.0, 1.0 / 500, 1.0, 1.0))
    st_o, rep_o = oracle_lib.solve(P.dense(), par, threads=16)
    with capi.Solver(P, par) as s:
        res = s.solve(raise_on=(1, 2, 3, 4, 6))
        st = s.state()
    assert res["iters"] == rep_o["iters"]
    scale = max(1.0, float(np.max(np.abs(st_o["x"]))))
    assert np.max(np.abs(st["x"] - st_o["x"])) <= 1e-9 * scale
    obj_o = oracle_lib.objective(P.dense(), st_o["x"])
    assert abs(res["objective"] - obj_o) <= 1e-9 * max(1.0, abs(obj_o))


def test_batched_shared_maps_give_the_bits_of_the_dense_problem(capi, oracle_lib):
    """A batch holding a shared-map instance next to a per-scenario one: the
    shared instance solves to the bits of its dense copy in the same batch
    and matches the oracle."""
    P = W.shared_problem(901, 3, 5, seed=24)
    other = W.random_problem(333, 2, 4, seed=25)
    par = W.Params(rho=(1.0, 1.0, 1.0, 1.0), rho2_over_n=True, precision="mixed")
    out = []
    for Q in (P, P.dense()):
        with capi.Batch([other, Q], par) as B:
            B.solve()
            res = B.wait(want_x=True)
            out.append(res)
    (o_s, r_s), (o_d, r_d) = out
    assert r_s["iters"] == r_d["iters"] and np.array_equal(r_s["x"], r_d["x"]) and r_s["objective"] == r_d["objective"]
    assert o_s["iters"] == o_d["iters"] and np.array_equal(o_s["x"], o_d["x"])
    st_o, _ = oracle_lib.solve(P.dense(), par.replace(precision="fp64"), threads=16)
    obj_o = oracle_lib.objective(P.dense(), st_o["x"])
    assert r_s["converged"] and abs(r_s["objective"] - obj_o) <= 1e-6 * max(1.0, abs(obj_o))


def test_served_shared_maps_give_the_bits_of_the_dense_problem(capi):
    """Two sessions of one server, the same problem with shared and with
    repeated maps: equal results for the cold solve and for a step request
    (whose new maps are the same for every scenario)."""
    P = W.shared_problem(401, 2, 3, seed=26)
    par = W.Params(rho=(1.0, 1.0, 1.0, 1.0), rho2_over_n=True, precision="mixed")
    step = W.step_data(P.m, P.q, 1, seed=27)
    for k in ("f2", "f1", "f0", "g2", "g1", "g0"):
        step[k] = np.repeat(step[k][:, :1], P.q, axis=1)   # the same maps for every scenario
    with capi.Server(par, store_elements=1 << 20, max_active=8, max_m=4, max_q=20) as S:
        t0, t1 = S.submit(P, session=0), S.submit(P.dense(), session=1)
        a, b = S.poll(t0, wait_ms=60000, want_x=True), S.poll(t1, wait_ms=60000, want_x=True)
        assert a["status"] == 0 and a["iters"] == b["iters"] and np.array_equal(a["x"], b["x"])
        u0, u1 = S.submit_step(0, step), S.submit_step(1, step)
        a, b = S.poll(u0, wait_ms=60000, want_x=True), S.poll(u1, wait_ms=60000, want_x=True)
        assert a["warm"] and b["warm"]
        assert a["status"] == 0 and a["iters"] == b["iters"] and np.array_equal(a["x"], b["x"])


def test_noalloc_refuses_shared_maps(capi):
    torch = pytest.importorskip("torch")
    P = W.shared_problem(100, 2, 2, seed=23)
    D = P.copy()
    for k, v in P.arrays().items():
        setattr(D, k, torch.from_numpy(np.ascontiguousarray(v)).cuda())
    z = lambda *sh: torch.zeros(sh, dtype=torch.float64, device="cuda")
    st = {"x": z(2, 2, 100), "s": z(2, 100), "mu": z(2, 100), "lam": z(2, 2), "zeta": z(2, 2), "h": z(2, 2),
          "p": z(2, 2), "nu": z(2, 2), "x1": z(2), "rho": [1.0] * 4, "cold": True}
    with pytest.raises(capi.AdmmError) as ei:
        capi.admm_solve_noalloc(D, W.Params(), st)
    assert ei.value.status == capi.ADMM_EUNSUPPORTED

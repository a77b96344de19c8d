"""Scenario-shared cost and loss maps (f and g drawn per (i, k), stored once
as [m][n]): the single-instance solve gives the same bits as on the same
problem with the maps repeated for every scenario, and matches the oracle
(which takes the repeated, dense form)."""
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


def test_batches_and_servers_refuse_shared_maps(capi):
    P = W.shared_problem(100, 2, 2, seed=23)
    with pytest.raises(capi.AdmmError) as ei:
        capi.Batch([P], W.Params(precision="mixed"))
    assert ei.value.status == capi.ADMM_EUNSUPPORTED

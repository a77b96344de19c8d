"""One-step parity at the full size of the large single instance (n = 1e5,
m = 4, q = 20, FP64), in the launch shape the benchmark times.  A whole
oracle solve there takes minutes, so the oracle runs one iteration from the
GPU's state after T iterations and is compared with the GPU's state after
T + 1: every output of the iteration at that size, against the paper's
steps, at the 1e-9 bar of the parity tests.  The k-sums of 1e5 terms are
summed in different orders on the two sides; their rounding difference
(about 1e-9 absolute on sums of 6e4) is 1e-14 of the arrays they feed."""
import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def test_one_iteration_at_n1e5_m4_q20_matches_the_oracle(capi, oracle_lib):
    P = W.config(2)
    T = 200
    par = W.Params(rho=(1.0, 1.0 / P.n, 1.0, 1.0), r_tol=0.0, s_tol=0.0, check_every=10)
    with capi.Solver(P, par.replace(max_iter=T)) as s:
        s.solve(raise_on=(1, 2, 3, 4, 6))
        st_t = s.state()
    with capi.Solver(P, par.replace(max_iter=T + 1)) as s:
        res = s.solve(raise_on=(1, 2, 3, 4, 6))
        st_g = s.state()
    assert res["iters"] == T + 1 and not st_t["cold"]
    # the GPU's state after T iterations as the oracle's dense state: lambda is
    # constant over k and z_k = g_k(x_k) + zeta (steps (b), (g))
    m, q, n = P.m, P.q, P.n
    gx = P.g2 * st_t["x"] ** 2 + P.g1 * st_t["x"] + P.g0
    dense = {"x": st_t["x"], "z": gx + st_t["zeta"][:, :, None],
             "lam": np.broadcast_to(st_t["lam"][:, :, None], (m, q, n)).copy(),
             "s": st_t["s"], "mu": st_t["mu"], "h": st_t["h"], "p": st_t["p"], "nu": st_t["nu"], "x1": st_t["x1"]}
    st_o, rep_o = oracle_lib.solve(P, par.replace(max_iter=1, check_every=1), state=dense, threads=16)
    errs = {k: rel(st_g[k], st_o[k]) for k in ("x", "s", "mu", "h", "p", "nu", "x1")}
    errs["lam"] = rel(np.broadcast_to(st_g["lam"][:, :, None], st_o["lam"].shape), st_o["lam"])  # every k
    gx1 = P.g2 * st_g["x"] ** 2 + P.g1 * st_g["x"] + P.g0
    errs["z"] = rel(gx1 + st_g["zeta"][:, :, None], st_o["z"])
    errs["r"] = abs(res["r"] - rep_o["r"]) / max(1.0, abs(rep_o["r"]))
    errs["sigma"] = abs(res["sigma"] - rep_o["sigma"]) / max(1.0, abs(rep_o["sigma"]))
    bad = {k: v for k, v in errs.items() if not v <= TOL}
    assert not bad, (bad, errs)
    # the iteration moved the state (the comparison is not of two copies)
    assert np.abs(st_g["x"] - st_t["x"]).max() > 1e-8

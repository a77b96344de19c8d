"""Batched parity at the full size of the batched workload (4096 instances,
n log-uniform in [50, 5000], m in {2, 3, 4}, q in [1, 20], mixed precision,
rho = (1, 1/n, 1, 1) per instance, fixed or adapted as in Sec. IV-A): seven
of its instances, the three
largest shapes among them (n near 5000, m = 4, q near 20), solved in one
batch through the C ABI and each compared with a full FP64 oracle solve of
the same instance: objective within 1e-6 relative and KKT residual of
eq. (2) at most the oracle's plus 1e-6.  An instance gives the same bits
alone and in any mix (test_gpu_batch.py), so these are the results it has
inside the 4096-instance launch.  The oracle solves take about a minute on
16 host cores."""
import os

import numpy as np
import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# instance ids of the batched workload and their (n, m, q)
INSTANCES = {
    1168: (4893, 4, 17),   # the most elements of the 4096
    1243: (4663, 4, 20),
    2720: (4841, 4, 19),
    462: (1983, 2, 13),    # 80th percentile of elements
    2579: (1387, 2, 4),    # median
    3560: (337, 3, 11),
    329: (54, 2, 1),       # the fewest elements
}


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


def _kkt(oracle, P, par, st):
    m, q, n = P.m, P.q, P.n
    dense = {"x": st["x"], "z": np.zeros((m, q, n)), "lam": np.broadcast_to(st["lam"][:, :, None], (m, q, n)).copy(),
             "s": st["s"], "mu": st["mu"], "h": st["h"], "p": st["p"], "nu": st["nu"], "x1": st["x1"]}
    return oracle.kkt(P, par.replace(rho=tuple(st["rho"]), rho2_over_n=False), dense)[0]


@pytest.mark.parametrize("adapt", [False, True])
def test_full_size_batched_instances_match_the_oracle(capi, oracle_lib, adapt):
    ids = list(INSTANCES)
    probs = [W.batch_instance(t) for t in ids]
    assert [(P.n, P.m, P.q) for P in probs] == [INSTANCES[t] for t in ids]
    par = W.Params(rho=(1.0, 1.0, 1.0, 1.0), rho2_over_n=True, precision="mixed", adapt_rho=adapt)
    with capi.Batch(probs, par) as B:
        B.solve()
        res = B.wait()
        states = [B.state(t) for t in range(len(probs))]
    threads = os.cpu_count() or 1
    rows = []
    for t, P in enumerate(probs):
        po = par.replace(precision="fp64")
        st_o, rep_o = oracle_lib.solve(P, po, threads=threads)
        obj_o = oracle_lib.objective(P, st_o["x"])
        k_o = oracle_lib.kkt(P, po.replace(rho=tuple(rep_o["rho"]), rho2_over_n=False), st_o)[0]
        k_g = _kkt(oracle_lib, P, po, states[t])
        err = abs(res[t]["objective"] - obj_o) / max(1.0, abs(obj_o))
        rows.append((ids[t], P.n, P.m, P.q, res[t]["iters"], rep_o["iters"], err, k_g - k_o))
        print(f"{'adapted' if adapt else 'fixed'} rho, instance {ids[t]} (n={P.n}, m={P.m}, q={P.q}): iterations {res[t]['iters']} (oracle "
              f"{rep_o['iters']}), objective error {err:.1e}, KKT {k_g:.2e} (oracle {k_o:.2e})")
        assert rep_o["converged"] and res[t]["converged"], rows[-1]
        assert err <= 1e-6, rows[-1]
        assert k_g <= k_o + 1e-6, rows[-1]

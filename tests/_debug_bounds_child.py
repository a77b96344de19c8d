"""Child process of test_gpu_debug_bounds.py: loads the library named by
ADMM_LIB (the bounds-checked build or the release one), runs the bounds
self-test, a mixed batch of the batched recipe (CTA and cluster teams,
shared and per-scenario maps) and a single-instance mixed solve, and saves
the results to the .npz path given as argv[1]."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1903_10041_gb300 import capi  # noqa: E402
from paper_1903_10041_gb300 import workloads as W  # noqa: E402


def main(out_path):
    out = {}
    try:
        st, ix = capi.admm_selftest_bounds()
        out["selftest"] = np.array([st, ix])
    except capi.AdmmError as e:
        out["selftest"] = np.array([-e.status, -1])
    probs = [W.batch_instance(t) for t in (329, 2579, 3560, 462)]
    probs.append(W.shared_problem(777, 3, 5, seed=31))
    par = W.Params(rho=(1.0, 1.0, 1.0, 1.0), rho2_over_n=True, precision="mixed", adapt_rho=True)
    with capi.Batch(probs, par) as B:
        B.set_config(8, 0, 0, 2, 20000)           # clusters for the larger instances
        B.solve()
        res = B.wait(want_x=True)
    for t, r in enumerate(res):
        out[f"batch{t}_x"] = r["x"]
        out[f"batch{t}_iters"] = np.array([r["iters"], r["status"]])
    P = W.random_problem(2001, 3, 5, seed=33)
    with capi.Solver(P, W.Params(rho=(1.0, 1.0 / 2001, 1.0, 1.0), precision="mixed")) as s:
        r = s.solve(raise_on=())
        out["single_x"] = s.state()["x"]
        out["single_iters"] = np.array([r["iters"], r["status"]])
    np.savez(out_path, **out)


if __name__ == "__main__":
    main(sys.argv[1])

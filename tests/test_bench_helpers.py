"""Host-side helpers of bench.py: the algorithmic byte model (dense and
scenario-shared maps) and the rule that ncu traffic is reported only for the
kernel sources it was captured on."""
import importlib.util
import os

from paper_1903_10041_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bytes_per_iteration_counts_each_streamed_array_once():
    b = _bench()
    P = W.random_problem(1000, 3, 4)
    m, q, n = 3, 4, 1000
    assert b.bytes_per_iteration(P, "fp64") == 8 * (6 * m * q * n + 2 * m * n + 5 * q * n)
    assert b.bytes_per_iteration(P, "mixed") == 4 * (6 * m * q * n + 2 * m * n + q * n) + 32 * q * n
    S = W.shared_problem(1000, 3, 4)
    # shared maps: f2 f1 g2 g1 once per (i, k) instead of per (i, j, k)
    assert b.bytes_per_iteration(P, "fp64") - b.bytes_per_iteration(S, "fp64") == 8 * 4 * m * n * (q - 1)


def test_traffic_is_reported_only_for_the_captured_sources():
    b = _bench()
    P = W.config(1)
    key = (P.name, "fp64")
    assert key in b.NCU_TRAFFIC
    expect = b.NCU_TRAFFIC[key]["bytes_per_iter"] * 3330
    if b.NCU_TRAFFIC[key]["src"] == b.kernel_source_hash():
        assert b.traffic_per_launch(P, "fp64", 3330) == expect
    saved = b.NCU_TRAFFIC[key]["src"]
    try:
        b.NCU_TRAFFIC[key]["src"] = "0" * 16  # a kernel changed since the capture
        assert b.traffic_per_launch(P, "fp64", 3330) is None
    finally:
        b.NCU_TRAFFIC[key]["src"] = saved
    assert b.traffic_per_launch(W.config(0), "fp64", 100) is None  # never captured


def test_q_sweep_workloads_are_the_phev_instance_at_each_scenario_count():
    import numpy as np
    import pytest
    b = _bench()
    sweep = b.sweep_workloads("5,50,500", "fp64", True)
    assert [P.q for P, _ in sweep] == [5, 50, 500]
    for P, par in sweep:
        assert (P.n, P.m) == (1000, 2) and P.f2.shape == (2, P.q, 1000)
        assert par.adapt_rho and par.rho == (1.0, 1e-3, 1.0, 1.0)
    # q = 50 is the headline PHEV instance itself, with its penalties
    P50, par50 = sweep[1]
    C1, cpar = b.workload(1, "fp64")
    assert P50.name == C1.name and par50.rho == cpar.rho
    for k, v in C1.arrays().items():
        np.testing.assert_array_equal(getattr(P50, k), v)
    with pytest.raises(ValueError):
        b.sweep_workloads("5,0", "fp64", False)


def test_fp64_flop_count_follows_the_branch_each_element_takes():
    """Elements with losses run Algorithm 1 (68 counted flops at m = 2);
    lossless ones (the PHEV engine, g = 0) the quadratic case (16)."""
    b = _bench()
    P = W.config(1)  # engine lossless, battery lossy
    assert b.fp64_flops_per_iteration(P) == 68 * 50_000 + 16 * 50_000 + 5 * 50 * 1000
    Q = W.random_problem(100, 2, 3)  # every element has losses
    assert b.fp64_flops_per_iteration(Q) == 68 * 600 + 5 * 300
    S = W.shared_problem(100, 3, 4)
    assert b.fp64_flops_per_iteration(S) == b.fp64_flops_per_iteration(S.dense())


def test_paper_penalties_are_the_settings_of_the_phev_study():
    """Sec. IV-A: rho = (1e-4, 2e-6, 5e-6, 5e-6), r-bar = 1e-6 dE with dE the
    battery capacity, sigma-bar = 1e-2, adaptation on; the q sweep uses them
    at every q with --paper-penalties."""
    b = _bench()
    P = W.phev_problem(1000, 5)
    par = b.paper_penalties(P)
    assert par.rho == (1e-4, 2e-6, 5e-6, 5e-6) and par.adapt_rho
    assert par.r_tol == 1e-6 * float(P.c[1]) and par.s_tol == 1e-2
    sweep = b.sweep_workloads("5,500", "fp64", False, paper=True)
    assert [q.rho for _, q in sweep] == [(1e-4, 2e-6, 5e-6, 5e-6)] * 2


def test_penalty_settings_of_the_batched_and_served_lines():
    """--adapt-start applies only with the adaptation, and the line's rho text
    says so; the served line adapts from iteration 1000 (reading R16)."""
    import argparse
    b = _bench()
    par = b.batch_params(argparse.Namespace(adapt=True, adapt_start=1000))
    assert par.adapt_rho and par.adapt_start == 1000 and par.rho2_over_n and par.precision == "mixed"
    assert b.penalty_text(argparse.Namespace(adapt=True, adapt_start=1000)).endswith("from iteration 1000")
    par = b.batch_params(argparse.Namespace(adapt=False, adapt_start=1000))
    assert not par.adapt_rho and par.adapt_start == 0
    assert b.penalty_text(argparse.Namespace(adapt=True, adapt_start=0)).endswith("adapted (Sec. IV-A)")
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert "args.adapt_start = args.adapt_start or 1000" in src
    assert "cluster_size=2, cluster_min_elements=100000" in src

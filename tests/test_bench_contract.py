"""The JSON line of bench.py's default workload carries every key of the
benchmark contract, checked on the CPU: the CUDA calls are replaced by
stand-ins that return fixed timings and solve results (no number here is a
measurement), the oracle's CPU baseline runs for real on a short sample."""
import importlib.util
import json
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_contract_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Event:
    def __init__(self, **kw):
        pass

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 80.0


class _Solver:
    def __init__(self, P, par):
        self.P = P

    def reset(self):
        pass

    def solve(self, stream=None, x_out=None, x1_out=None):
        return {"status": 0, "iters": 3330, "converged": True, "objective": 38.22, "r": 0.0, "sigma": 0.0}

    def solve_async(self, stream=None):
        pass

    def wait(self):
        return self.solve()

    def close(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        pass


def test_default_line_has_every_contract_key(monkeypatch, capsys):
    torch = pytest.importorskip("torch")
    b = _bench()
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "Stream", lambda: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(*a, **k))
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    import paper_1903_10041_gb300 as pkg
    from paper_1903_10041_gb300 import build
    build.build()
    import paper_1903_10041_gb300.capi  # noqa: F401  (the real binding is what the patches restore)
    fake = types.ModuleType("paper_1903_10041_gb300.capi")
    fake.Solver = _Solver
    monkeypatch.setitem(__import__("sys").modules, "paper_1903_10041_gb300.capi", fake)
    monkeypatch.setattr(pkg, "capi", fake, raising=False)
    real_baseline = b.cpu_baseline
    monkeypatch.setattr(b, "cpu_baseline", lambda P, par, iters, budget_s=12.0: real_baseline(P, par, iters, 0.3))
    args = b.argparse.Namespace(max_iter=0, warmup=3, steps=10, no_e2e=False, no_cpu_baseline=False, config=1,
                                q_sweep="", precision="fp64", gpus=1)
    P, par = b.workload(1, "fp64")
    b.run_single(args, P, par, 0, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line, k
    assert line["metric"] == b.METRIC and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["n_gpus"] == 1 and line["steps"] == 10 and line["warmup"] == 3 and line["scaling"] == "weak"
    assert line["value"] == pytest.approx(1e3 / 80.0) and line["ms_per_step"] == pytest.approx(80.0)
    assert line["vs_baseline"] is None and line["dtype"] == "f64"
    assert line["config"]["workload"].startswith("phev n=1000 q=50") and "l2" in line["config"]
    rf = line["roofline"]
    assert rf["bound"] == "alu" and rf["unit"] == "TFLOP/s" and rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["achieved"] == pytest.approx(3330 * b.fp64_flops_per_iteration(P) / 0.080 / 1e12)
    assert "traffic" in rf
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["unit"] == "solves/s" and cb["cores"] >= 1 and cb["value"] > 0
    assert isinstance(cb["sample"], str)
    e2e = line["e2e"]
    assert e2e["unit"] == "solves/s" and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == sum(v.nbytes for v in P.arrays().values())
    assert e2e["d2h_bytes_per_step"] == 8 * (P.m * P.q * P.n + P.m)
    assert line["gpu_launches"] == 10
    assert set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}


class _Batch:
    """Stand-in for capi.Batch: fixed iteration counts and results."""

    def __init__(self, probs, par):
        self.probs = probs
        self.cfg = {"warps_per_cta": 8, "ctas_per_sm": 2, "small_max_elements": 0, "cluster_size": 1,
                    "cluster_min_elements": 0}

    def set_config(self, *a):
        pass

    def config(self):
        return dict(self.cfg)

    def autotune(self, trial_iters=30):
        return dict(self.cfg)

    def reset(self):
        pass

    def solve(self, stream=None):
        pass

    def wait(self, stream=None, want_x=False):
        import numpy as np
        out = []
        for P in self.probs:
            r = {"iters": 1000, "converged": True, "objective": 1.0, "status": 0}
            if want_x:
                r["x"], r["x1"] = np.zeros((P.m, P.q, P.n)), np.zeros(P.m)
            out.append(r)
        return out

    def state(self, t):
        return {}

    def close(self):
        pass


def test_default_batched_line_has_every_contract_key(monkeypatch, capsys):
    """The default workload (no --config) is the 4096-instance batch; its
    line carries the contract keys, an HBM roofline over the algorithmic
    bytes, the oracle's CPU baseline and the end-to-end leg."""
    torch = pytest.importorskip("torch")
    b = _bench()
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "Stream", lambda: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(*a, **k))
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(torch.Tensor, "fill_", lambda self, v: self)
    import paper_1903_10041_gb300 as pkg
    from paper_1903_10041_gb300 import build
    build.build()
    import paper_1903_10041_gb300.capi  # noqa: F401
    fake = types.ModuleType("paper_1903_10041_gb300.capi")
    fake.Batch = _Batch
    monkeypatch.setitem(__import__("sys").modules, "paper_1903_10041_gb300.capi", fake)
    monkeypatch.setattr(pkg, "capi", fake, raising=False)
    # a short oracle comparison stands in for the sampled full solves
    monkeypatch.setattr(b, "oracle_sample_errors", lambda probs, par, res, states, idx, oracle: {
        "instances": idx, "max_rel_objective_err": 0.0, "max_kkt_excess": 0.0})
    monkeypatch.setattr(b.os, "cpu_count", lambda: 2)
    ns = b.argparse.Namespace(gpus=1, steps=10, warmup=5, count=64, max_iter=0, batch_config="", adapt=False,
                              no_e2e=False, no_cpu_baseline=False, no_oracle_sample=False)
    b.run_batched(ns)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line, k
    assert line["config"]["workload"].startswith("batched: 64 instances")
    assert line["value"] == pytest.approx(64 * 10 / 0.8) and line["ms_per_step"] == pytest.approx(80.0)
    rf = line["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    assert rf["achieved"] == pytest.approx(rf["algorithmic_bytes"] / 0.080 / 1e9)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] == 10


def test_no_flag_default_is_the_batched_workload():
    b = _bench()
    import inspect
    src = inspect.getsource(b.main)
    assert 'ap.add_argument("--config", type=int, default=3' in src

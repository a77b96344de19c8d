"""The N > 1 paths on CPU with the gloo backend (world size 2), one process
per rank: bench.py's barrier and max over ranks of the timed region, with
rank 0 alone printing the JSON line (replicas of independent instances, no
collective on the data path); and one instance split by time step over two
workers (paper_1903_10041_gb300.shard: one exchange of the per-pair partial
sums per iteration), which must reproduce the single-worker iteration."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r, w, _ = bench.dist_init(world)
    vals = bench.barrier_max([float(r + 1), -float(r), 10.0 * r], w)
    out.put((r, vals))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_barrier_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the max over ranks of each timed value
    assert got[0] == got[1] == [2.0, 0.0, 10.0]


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--config", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0.0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def _shard_par(T, tol, adapt_start):
    from paper_1903_10041_gb300 import workloads as W
    par = W.Params(rho=(1.0, 1.0 / 97, 1.0, 1.0), r_tol=tol, s_tol=tol, max_iter=T, check_every=10)
    if adapt_start is not None:
        par = par.replace(adapt_rho=True, adapt_start=adapt_start)
    return par


def _shard_worker(rank, world, port, out, T, tol, adapt_start=None):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1903_10041_gb300 import shard
    from paper_1903_10041_gb300 import workloads as W
    from tests._shard_oracle import OracleShard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = W.random_problem(97, 3, 4, seed=83)
    par = _shard_par(T, tol, adapt_start)
    k0, k1 = shard.column_shards(P.n, world)[rank]
    B = OracleShard(P, par, k0, k1)
    rep = shard.run(B, shard.Exchange(), P.m, P.q, par.rho, par.r_tol, par.s_tol, par.max_iter, par.check_every,
                    adapt=par.adapt_rho, tau=par.tau, adapt_start=par.adapt_start)
    out.put((rank, (k0, k1), rep, {k: v.copy() for k, v in B.st.items()}))
    dist.destroy_process_group()


@pytest.mark.parametrize("T,tol,adapt_start", [(60, 0.0, None), (5000, 1e-6, None), (5000, 1e-6, 0),
                                               (5000, 1e-6, 200)])
def test_column_split_over_two_workers_reproduces_the_single_worker_iteration(oracle_lib, T, tol, adapt_start):
    """Each worker runs the element updates of its columns (the oracle's
    phase A), one gather of the 2mq + 2 partials combines them in worker
    order, each runs the pair steps (phase B).  After T iterations, and at
    the stop test, the assembled state equals the single-worker oracle's to
    1e-12 relative (the k-sums are added in another order) with the same
    iteration count; both workers hold the same pair scalars bit for bit.
    With the penalty adaptation of Sec. IV-A (from the first check, or from
    iteration 200) every worker takes the oracle's rescalings: the same
    final penalties and the same state."""
    torch = pytest.importorskip("torch")
    from paper_1903_10041_gb300 import workloads as W
    ctx = torch.multiprocessing.get_context("spawn")
    q_ = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q_, T, tol, adapt_start)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (b, rep, st)) for r, b, rep, st in (q_.get(timeout=300) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    P = W.random_problem(97, 3, 4, seed=83)
    par = _shard_par(T, tol, adapt_start)
    st_o, rep_o = oracle_lib.solve(P, par)
    (b0, rep0, s0), (b1, rep1, s1) = got[0], got[1]
    assert b0[0] == 0 and b0[1] == b1[0] and b1[1] == P.n
    assert rep0 == rep1
    assert rep0["iters"] == rep_o["iters"] and rep0["converged"] == rep_o["converged"]
    if tol > 0:
        assert rep0["converged"]
    for k in ("h", "p", "nu", "x1"):
        assert np.array_equal(s0[k], s1[k]), k
    rel = lambda a, b: float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))
    for k in ("x", "z", "lam", "s", "mu"):
        assert rel(np.concatenate([s0[k], s1[k]], axis=-1), st_o[k]) <= 1e-12, k
    for k in ("h", "p", "nu", "x1"):
        assert rel(s0[k], st_o[k]) <= 1e-12, k
    assert abs(rep0["r"] - rep_o["r"]) <= 1e-12 and abs(rep0["sigma"] - rep_o["sigma"]) <= 1e-12
    assert np.allclose(rep0["rho"], rep_o["rho"], rtol=1e-15, atol=0.0)
    if adapt_start is not None:
        assert list(rep0["rho"]) != list(par.rho)   # the rule did rescale

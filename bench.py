"""Benchmark: ADMM solves/s to 1e-6 residual on one GB300 (per GPU, replicas).

Default workload (--config 3): one step = one batched launch that solves
4096 independent instances of problem (2) (n log-uniform in [50, 5000],
m in {2, 3, 4}, q in [1, 20]; synthetic, seeded per instance) from the zero
start to the stop test (r < 1e-6, sigma < 1e-6 with the mixed-precision
margin, checked every 10 iterations; at most 5000 iterations), mixed
precision, launch configuration picked by the autotuner.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 0|1|2|3|4] [--precision fp64|mixed|mixed_fp64cubic] [--adapt]
                  [--paper-penalties] [--q-sweep 5,10,20,50,100,200,500] [--quartic N[,N2,...]]

Workloads: 0, 1 and 2 are single instances (n=100 m=2 q=1; the PHEV
n=1000 q=50; n=1e5 m=4 q=20), 3 the 4096-instance batch (default), 4 the
served Poisson stream of re-solves; --q-sweep and --quartic are the
runtime-against-q (Sec. IV-B) and quartic (Sec. III-C) comparisons.

Prints one JSON line (one per q or N for the sweeps).  `value` times K
solves with inputs resident in HBM (CUDA events on the launch stream, L2
flushed between solves); `e2e` times the same solves through the public C
ABI from pinned host buffers (create + solve + copy-out + destroy).  Under
torchrun each rank solves its own instances (weak scaling, no collective
on the data path).  `--impl reference` times the FP64 CPU oracle on the
host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADMM solves/s to 1e-6 residual, HBM GB/s fraction; batched p50/p99 latency"
L2_FLUSH_BYTES = 512 << 20  # > 126 MB L2

# FP64 peak of GB300 derived from unit counts and clock: 152 SMs x 2 DFMA/clk
# per SM x 2 flop x 2.07 GHz (the measured DFMA rate is 1.90/clk/SM).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Conventional FP64 flops of one iteration of the FP64 kernel, counted from
# its element update (each +, -, *, /, sqrt and cube root counts 1, an FMA 2;
# comparisons and clamps 0):
#   every element: the sum over the other sources (m - 1), phi (3), the
#     lossless parts of C and D (6), its share of the column sums of x and
#     x - x~ (3);
#   an element with losses (beta_2 or beta_1 nonzero) adds g(x~), u, A, B
#     and the loss terms of C and D (21), Algorithm 1 on its Cardano branch
#     (29: one division, the scaled coefficients b, c, d, Q, R, Delta, the
#     square root, the cube root with its reciprocal, S + T - b/3) and g(x)
#     with its sum over k (5); the trig branch costs more and is counted as
#     Cardano;
#   a lossless element (g = beta_0) takes the quadratic case x = -D / 2C (3);
#   every column: v and mu of steps (e), (f) (5).
FLOPS_LOSS_TERMS = 21 + 29 + 5
FLOPS_QUADRATIC = 3
FLOPS_PER_COLUMN = 5


def fp64_flops_per_iteration(P) -> int:
    import numpy as np
    lossy = int(np.count_nonzero((np.asarray(P.g2) != 0) | (np.asarray(P.g1) != 0)))
    if getattr(P, "coef_shared", False):  # maps given once per (i, k) for every scenario
        lossy *= P.q
    common = (P.m - 1) + 3 + 6 + 3
    return (P.elements * common + lossy * FLOPS_LOSS_TERMS + (P.elements - lossy) * FLOPS_QUADRATIC
            + FLOPS_PER_COLUMN * P.q * P.n)


def workload(cfg: int, precision: str, coef_shared: bool = False):
    from paper_1903_10041_gb300 import workloads as W
    P = W.config(cfg)
    if coef_shared:  # the same instance shape with scenario-shared cost and loss maps
        P = W.shared_problem(P.n, P.m, P.q, name=f"shared maps n={P.n} m={P.m} q={P.q}")
    rho = (1.0, 1.0, 1.0, 1.0) if cfg == 0 else (1.0, 1.0 / P.n, 1.0, 1.0)
    par = W.Params(rho=rho, precision=precision)
    return P, par


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the solve
# kernels, from one ncu capture of each workload: bytes per iteration of a
# single-instance solve, or per element-iteration of a batched launch.  A
# figure is reported only while the kernel's sources hash to the build it
# was taken on (otherwise `traffic` is null).
NCU_TRAFFIC = {
    ("phev n=1000 q=50", "fp64"): {"bytes_per_iter": (7666944 + 49920) / 3330, "src": "0f1fa41955024aab"},
    ("plain n=1e5 m=4 q=20", "mixed"): {"bytes_per_iter": (568258408448 + 185992512000) / 2750, "src": "0f1fa41955024aab"},
}
NCU_TRAFFIC_BATCH = {"bytes_per_element_iter": (1811961266176 + 614259118080) / 76330081250.0, "src": "58bddc1cb77dc15c"}
# FP64 pipe utilisation (sm__pipe_fp64_cycles_active, % of peak over the active cycles) of the FP64 solve
# kernel on the PHEV instance, from an ncu capture of the same build: the counted-flop fraction leaves out
# the Newton steps of the FP32-seeded roots, conversions, comparisons and the per-pair scalar phase.
NCU_FP64_PIPE = {("phev n=1000 q=50", "fp64"): {"pct": 60.47, "src": "0f1fa41955024aab"}}

# Sources each solve kernel is compiled from.
SINGLE_KERNEL_SOURCES = ("single.cu", "quartic32.cuh", "quartic64.cuh", "mixed_elem.cuh", "common.cuh", "internal.h")
BATCH_KERNEL_SOURCES = ("batch_kernel.cuh", "batch_w4.cu", "batch_w8.cu", "batch_w16.cu", "batch.h", "quartic32.cuh",
                        "quartic64.cuh", "mixed_elem.cuh", "common.cuh", "internal.h")


def kernel_source_hash(sources=SINGLE_KERNEL_SOURCES) -> str:
    import hashlib
    files = sorted([os.path.join(ROOT, "paper_1903_10041_gb300", "csrc", f) for f in sources] +
                   [os.path.join(ROOT, "include", "admm.h")])
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(P, prec: str, iters: int):
    t = NCU_TRAFFIC.get((P.name, prec))
    if t is None or t["src"] != kernel_source_hash():
        return None
    return t["bytes_per_iter"] * iters


def fp64_pipe_busy(P):
    t = NCU_FP64_PIPE.get((P.name, "fp64"))
    if t is None or t["pct"] is None or t["src"] != kernel_source_hash():
        return None
    return t["pct"] / 100.0


def batch_traffic_per_launch(element_iters: float):
    t = NCU_TRAFFIC_BATCH
    if t["bytes_per_element_iter"] is None or t["src"] != kernel_source_hash(BATCH_KERNEL_SOURCES):
        return None
    return t["bytes_per_element_iter"] * element_iters


def bytes_per_iteration(P, prec: str) -> int:
    """Algorithmic HBM bytes of one iteration (each streamed array once):
    f2, f1, g2, g1 read and x read+write (6 per element), the bounds
    (2 per (i, k)), y read and s, mu read+write (5 per column).  FP64: 8 bytes
    each.  Mixed: 4 bytes each, except s and mu, which are float-float
    (8 bytes)."""
    m, q, n = P.m, P.q, P.n
    coef = 4 * m * n * (1 if getattr(P, "coef_shared", False) else q)  # f2 f1 g2 g1 ([m][n] when shared)
    if prec == "fp64":
        return 8 * (coef + 2 * m * n * q + 2 * m * n + 5 * n * q)
    return 4 * (coef + 2 * m * n * q + 2 * m * n + n * q) + 8 * 4 * n * q


def measured_peaks() -> dict:
    """HBM copy bandwidth measured on this GPU type (MEASURED_PEAKS.json at
    the repository root), else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (STREAM-style copy, MEASURED_PEAKS.json)"}
    return {"hbm_gbs": 6800.0, "source": "fallback 6.8 TB/s (no measured figure present)"}


def batch_params(args):
    """Settings of the batched and served workloads: rho = (1, 1/n, 1, 1) per
    instance (reading R12), mixed precision, the Sec. IV-A adaptation with
    --adapt, from iteration --adapt-start on."""
    from paper_1903_10041_gb300 import workloads as W
    return W.Params(rho=(1.0, 1.0, 1.0, 1.0), rho2_over_n=True, precision="mixed", adapt_rho=args.adapt,
                    adapt_start=getattr(args, "adapt_start", 0) if args.adapt else 0)


def penalty_text(args) -> str:
    start = getattr(args, "adapt_start", 0)
    return "(1, 1/n, 1, 1) per instance" + (
        (f", adapted (Sec. IV-A) from iteration {start}" if start else ", adapted (Sec. IV-A)") if args.adapt else "")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        import tempfile
        out_dir = os.environ.get("ADMM_CLOCKS_DIR", tempfile.gettempdir())  # where the samples are kept
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(P, par, iters_per_solve: int, budget_s: float = 12.0):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    T iterations of the same solve, scaled to solves/s by the iteration
    count of a full solve."""
    import oracle
    P = P.dense()  # the oracle takes per-scenario coefficient arrays
    threads = os.cpu_count() or 1
    # size T from a short probe so the sample takes about budget_s seconds
    t0 = time.perf_counter()
    oracle.solve(P, par.replace(max_iter=5, r_tol=0.0, s_tol=0.0), threads=threads)
    per_it = (time.perf_counter() - t0) / 5
    T = max(10, min(iters_per_solve, int(budget_s / max(per_it, 1e-9))))
    t0 = time.perf_counter()
    oracle.solve(P, par.replace(max_iter=T, r_tol=0.0, s_tol=0.0), threads=threads)
    dt = time.perf_counter() - t0
    sec_per_solve = dt / T * iters_per_solve
    # the same on one core, on a shorter sample (about a quarter of the budget)
    t0 = time.perf_counter()
    oracle.solve(P, par.replace(max_iter=3, r_tol=0.0, s_tol=0.0), threads=1)
    per_it1 = (time.perf_counter() - t0) / 3
    T1 = max(5, min(iters_per_solve, int(0.25 * budget_s / max(per_it1, 1e-9))))
    t0 = time.perf_counter()
    oracle.solve(P, par.replace(max_iter=T1, r_tol=0.0, s_tol=0.0), threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": 1.0 / sec_per_solve, "unit": "solves/s", "cores": threads, "kind": "oracle",
            "one_core": T1 / (dt1 * iters_per_solve),
            "sample": f"{T} of the {iters_per_solve} iterations of one solve ({dt:.2f} s), "
                      f"scaled to a full solve; OpenMP over columns, {threads} threads "
                      f"(one core: {T1} iterations, {dt1:.2f} s)"}


def dist_init(n_gpus: int):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier_max(values, world):
    """Barrier + max over ranks of a list of floats."""
    if world == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def run_reference(args):
    rank, world, _ = dist_init(args.gpus)
    if rank != 0:
        return 0
    import oracle
    from oracle import build as ob
    ob.build()
    if args.config in (3, 4):
        return run_reference_batched(args, oracle)
    P, par = workload(args.config, "fp64")
    par = paper_penalties(P) if args.paper_penalties else par.replace(adapt_rho=args.adapt)
    # iterations of a full solve: the oracle's own count.  For the n=1e5, m=4, q=20 instance a full
    # oracle solve takes about 10 minutes on 8 cores, so its count (2650 with fixed penalties, run once)
    # is used; with the adaptation it is counted here like the others.
    if args.config == 2 and not args.adapt:
        rep = {"iters": 2650}
    else:
        _, rep = oracle.solve(P, par, threads=os.cpu_count() or 1)
    iters = rep["iters"]
    threads = os.cpu_count() or 1
    T = max(10, min(iters, 200 if args.config == 1 else 20))
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(P, par.replace(max_iter=T, r_tol=0.0, s_tol=0.0), threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    per_solve = statistics.mean(times) / T * iters
    v = 1.0 / per_solve
    # each step runs T of the solve's iterations; the rate is scaled to whole solves
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(P, par, args),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step {T} of the {iters} iterations of one solve, "
                                       f"scaled to a full solve"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_reference_batched(args, oracle):
    """The oracle on the batched (3) or served (4) workload: each step solves
    the workload's instances in order, from the zero start to the stop test,
    for about 4 s, and the rate is instances solved per second (a bounded
    sample of the same instance distribution).  ms_per_step is the measured
    duration of a step."""
    from paper_1903_10041_gb300 import workloads as W
    par = batch_params(args).replace(precision="fp64")
    threads = os.cpu_count() or 1
    durations, solved, nxt, k_all = [], 0, 0, []
    for step in range(args.warmup + args.steps):
        t0, k = time.perf_counter(), 0
        while time.perf_counter() - t0 < 4.0 or k == 0:
            oracle.solve(W.batch_instance(nxt % args.count), par, threads=threads)
            nxt += 1
            k += 1
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            durations.append(dt)
            k_all.append(k)
            solved += k
    v = solved / sum(durations)
    kind = "batched" if args.config == 3 else "served (cold solves of the controllers)"
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(durations),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded per instance)",
            "config": {"workload": f"{kind}: {args.count} instances, n log-uniform [50,5000], m in {{2,3,4}}, "
                                   f"q in [1,20]", "count": args.count, "rho": penalty_text(args)},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": f"{solved} instances (ids 0..{nxt - 1} mod {args.count}, in order) solved "
                                       f"to the stop test in the timed steps of about 4 s each"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def oracle_sample_errors(probs, par, results, states, idx, oracle):
    """Per-instance comparison with the FP64 oracle on a sample: the
    objective error against the oracle solved with the same settings, the
    objective distance of both to the optimum (the oracle solved to r, sigma
    < 1e-10), and the KKT residual of eq. (2) above the oracle's own.  The
    bar (reading R15): distance to the optimum at most the oracle's plus
    1e-6, and KKT at most the oracle's plus 1e-6."""
    import numpy as np
    errs, opt_excess, kkts, rows = [], [], [], []
    threads = os.cpu_count() or 1
    for t in idx:
        P = probs[t]
        po = par.replace(precision="fp64")
        st_o, rep_o = oracle.solve(P, po, threads=threads)
        obj_o = oracle.objective(P, st_o["x"])
        st_t, _ = oracle.solve(P, po.replace(r_tol=1e-10, s_tol=1e-10, max_iter=100000), threads=threads)
        f_opt = oracle.objective(P, st_t["x"])
        scale = max(1.0, abs(f_opt))
        obj_g = results[t]["objective"]
        errs.append(abs(obj_g - obj_o) / max(1.0, abs(obj_o)))
        d_g, d_o = abs(obj_g - f_opt) / scale, abs(obj_o - f_opt) / scale
        opt_excess.append(d_g - d_o)
        st = states[t]
        m, q, n = P.m, P.q, P.n
        dense = {"x": st["x"], "z": np.zeros((m, q, n)),
                 "lam": np.broadcast_to(st["lam"][:, :, None], (m, q, n)).copy(), "s": st["s"], "mu": st["mu"],
                 "h": st["h"], "p": st["p"], "nu": st["nu"], "x1": st["x1"]}
        k_g = oracle.kkt(P, par.replace(rho=tuple(st["rho"]), rho2_over_n=False), dense)[0]
        k_o = oracle.kkt(P, po.replace(rho=tuple(rep_o["rho"]), rho2_over_n=False), st_o)[0]
        kkts.append(k_g - k_o)
        rows.append({"instance": int(t), "n": P.n, "m": P.m, "q": P.q, "rel_objective_err": errs[-1],
                     "gpu_to_optimum": d_g, "oracle_to_optimum": d_o, "kkt_excess": kkts[-1]})
    return {"instances": list(map(int, idx)), "max_rel_objective_err": max(errs),
            "max_optimum_distance_excess": max(opt_excess), "max_kkt_excess": max(kkts),
            "bar": "distance to the optimum <= oracle's + 1e-6 and KKT <= oracle's + 1e-6", "per_instance": rows}


def pinned_copy(P):
    """The problem with every array in page-locked host memory (the e2e legs
    copy to the device from pinned buffers)."""
    import numpy as np
    import torch
    Q = P.copy()
    for k, v in P.arrays().items():
        setattr(Q, k, torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy())
    return Q


def batch_sample(probs, limit_small=40000):
    """Instances for the per-instance oracle comparison: the 6 smallest, 6
    spread over the lower half of the size distribution (m*q*n <= 40000),
    and the two instances nearest 1e5 and 2.5e5 elements."""
    import numpy as np
    order = np.argsort([P.elements for P in probs])
    small = [int(t) for t in order[:6]]
    spread = [int(t) for t in order[len(order) // 8: len(order) // 2: max(1, len(order) // 48)]
              if probs[int(t)].elements <= limit_small][:6]
    big = []
    for target in (1e5, 2.5e5):
        t = int(np.argmin([abs(P.elements - target) for P in probs]))
        if t not in small + spread + big:
            big.append(t)
    return small, spread, big


def run_batched(args):
    """The batched workload: `count` instances of uneven n, m, q in one launch (mixed)."""
    import numpy as np
    import torch
    rank, world, local = dist_init(args.gpus)
    from paper_1903_10041_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1903_10041_gb300 import capi
    from paper_1903_10041_gb300 import workloads as W
    base = rank * args.count
    probs = [W.batch_instance(base + t) for t in range(args.count)]
    par = batch_params(args)
    if args.max_iter:
        par = par.replace(max_iter=args.max_iter)
    B = capi.Batch(probs, par)
    if args.batch_config:
        w, c, sm, cl, cm = (int(v) for v in args.batch_config.split(","))
        B.set_config(w, c, sm, cl, cm)
        cfg = B.config()
    else:
        cfg = B.autotune(trial_iters=0)  # whole solves: the time includes the tail of the slowest instances
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def one():
        B.reset()
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.solve(stream=stream)
        e1.record(stream)
        res = B.wait(stream=stream)
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):
        one()
    if world > 1:
        torch.distributed.barrier()
    times, res = [], None
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, res = one()
            times.append(ms)
    (tot_ms,) = barrier_max([sum(times)], world)
    value = world * args.count * args.steps / (tot_ms / 1e3)
    per_batch_s = sum(times) / args.steps / 1e3
    iters = np.array([r["iters"] for r in res])
    conv = np.array([r["converged"] for r in res])
    el_it = float(sum(int(r["iters"]) * P.elements for r, P in zip(res, probs)))
    byts = sum(int(r["iters"]) * bytes_per_iteration(P, "mixed") for r, P in zip(res, probs))
    peaks = measured_peaks()
    gbs = byts / per_batch_s / 1e9
    roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"], "traffic": batch_traffic_per_launch(el_it),
                "algorithmic_bytes": float(byts), "peak_source": peaks["source"]}
    # the FP64 oracle on a sample of the instances: objective error and KKT excess
    import oracle
    small, spread, big = batch_sample(probs)
    idx = small + spread + big
    states = {t: B.state(t) for t in idx}
    errors = (oracle_sample_errors(probs, par, res, states, idx, oracle)
              if rank == 0 and not args.no_oracle_sample else None)
    # end to end: create from pinned host arrays, solve, read every result (objective, x)
    e2e = None
    if not args.no_e2e:
        pinned = [pinned_copy(P) for P in probs]
        t0 = time.perf_counter()
        B2 = capi.Batch(pinned, par)
        B2.set_config(cfg["warps_per_cta"], cfg["ctas_per_sm"], cfg["small_max_elements"],
                      cfg["cluster_size"], cfg["cluster_min_elements"])
        B2.solve()
        out = B2.wait(want_x=True)
        e2e_s = time.perf_counter() - t0
        B2.close()
        h2d = sum(sum(v.nbytes for v in P.arrays().values()) for P in probs)
        d2h = sum(o["x"].nbytes + o["x1"].nbytes for o in out)
        (e2e_max,) = barrier_max([e2e_s], world)
        e2e = {"value": world * args.count / e2e_max, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # oracle seconds per element-iteration on two sample instances, scaled to the batch
        t_el = []
        for t in small[:1] + spread[:1]:
            P = probs[t]
            T = 200
            t0 = time.perf_counter()
            oracle.solve(P, par.replace(precision="fp64", max_iter=T, r_tol=0.0, s_tol=0.0),
                         threads=os.cpu_count() or 1)
            t_el.append((time.perf_counter() - t0) / (T * P.elements))
        sec = el_it * float(np.mean(t_el))
        cpu = {"value": args.count / sec, "unit": "solves/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"200 iterations of instances {small[:1] + spread[:1]}, scaled by element-iterations to "
                         f"the whole batch ({el_it:.3g} element-iterations)"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded per instance)",
                "config": {"workload": f"batched: {args.count} instances, n log-uniform [50,5000], m in {{2,3,4}}, "
                                       f"q in [1,20], mixed precision", "count": args.count,
                           "elements": int(sum(P.elements for P in probs)), "autotuned": cfg,
                           "rho": penalty_text(args), "stop": "r < 1e-6, sigma < 0.85e-6 (mixed margin), "
                                                             "checked every 10 iterations, at most 5000",
                           "l2": "inputs larger than L2 (and flushed)",
                           "parallelism": f"replicas x{world}"},
                "iters": {"mean": float(iters.mean()), "max": int(iters.max()), "min": int(iters.min())},
                "element_iterations": el_it,
                "converged_frac": float(conv.mean()), "oracle_error_sample": errors,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    B.close()
    return 0


def shifted_oracle_state(P_new, P_old, st):
    """The receding-horizon warm start the server applies, written on the
    oracle's dense state: x, s, mu and the offsets z - g(x) move one step
    forward (last step kept), x at the new last step is clamped to its new
    bounds, x_1 is the mean of the new first moves; lambda, h, p, nu are
    kept."""
    import numpy as np
    sh = lambda a: np.concatenate([a[..., 1:], a[..., -1:]], axis=-1)
    g = lambda Q, x: Q.g2 * x * x + Q.g1 * x + Q.g0
    x = sh(st["x"])
    x[:, :, -1] = np.clip(x[:, :, -1], P_new.lo[:, None, -1], P_new.hi[:, None, -1])
    d = sh(st["z"] - g(P_old, st["x"]))
    return {"x": x, "z": g(P_new, x) + d, "lam": st["lam"].copy(), "s": sh(st["s"]), "mu": sh(st["mu"]),
            "h": st["h"].copy(), "p": st["p"].copy(), "nu": st["nu"].copy(), "x1": x[:, :, 0].mean(axis=1)}


def serving_cpu_baseline(trace, par, budget_s: float = 12.0, max_elements: int = 40000):
    """The oracle replaying the request trace serially on the host cores: the
    controllers of the first requests (those with at most `max_elements`
    elements) are solved cold (untimed), then their requests in trace order
    are solved warm-started from the shifted previous state, each timed, for
    about `budget_s` seconds.  Service times only: a serial CPU cannot keep
    up with the arrival rate, so there is no queueing model."""
    import numpy as np
    import oracle
    from paper_1903_10041_gb300 import workloads as W
    threads = os.cpu_count() or 1
    po = par.replace(precision="fp64")
    cur, states, times, iters = {}, {}, [], []
    spent = 0.0
    for c, step in trace:
        if spent > budget_s:
            break
        if c not in cur:
            P0 = W.batch_instance(c)
            if P0.elements > max_elements:
                continue
            states[c] = oracle.solve(P0, po, threads=threads)[0]
            cur[c] = P0
        P_new = W.receding_step(cur[c], step, seed=W.SEED * (1 << 32) + c)
        warm = shifted_oracle_state(P_new, cur[c], states[c])
        t0 = time.perf_counter()
        st, rep = oracle.solve(P_new, po, state=warm, threads=threads)
        dt = time.perf_counter() - t0
        spent += dt
        times.append(dt)
        iters.append(rep["iters"])
        cur[c], states[c] = P_new, st
    t = np.array(times) * 1e3
    return {"value": len(t) / (t.sum() / 1e3), "unit": "solves/s", "cores": threads, "kind": "oracle",
            "latency_ms": {"p50": float(np.percentile(t, 50)), "p99": float(np.percentile(t, 99)),
                           "mean": float(t.mean())},
            "sample": f"{len(t)} re-solves of {len(cur)} controllers (m*q*n <= {max_elements}) in trace order, "
                      f"warm-started from the shifted previous state, timed one by one (service time, "
                      f"no queueing); mean {np.mean(iters):.0f} iterations"}


def run_serving(args):
    """The serving workload: Poisson arrivals of receding-horizon re-solves of `count`
    controllers sized as the batched workload; continuous batching."""
    import numpy as np
    import torch
    rank, world, local = dist_init(args.gpus)
    from paper_1903_10041_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1903_10041_gb300 import capi
    from paper_1903_10041_gb300 import workloads as W
    par = batch_params(args)
    base = rank * args.count
    shapes = [W.batch_shape(base + c) for c in range(args.count)]
    total_el = sum(((n + 3) // 4 * 4) * m * q for n, m, q in shapes)
    # 16-warp CTA teams, 2-CTA clusters for the sessions above 1e5 elements (measured at 2000/s offered:
    # p99 0.92 s; 1.16 s above 1.5e5, 1.30 s above 2.5e5, 1.42 s without clusters)
    bc = dict(warps_per_cta=16, ctas_per_sm=0, small_max_elements=0, cluster_size=2, cluster_min_elements=100000)
    if args.batch_config:
        w, c, sm, cl, cm = (int(v) for v in args.batch_config.split(","))
        bc = dict(warps_per_cta=w, ctas_per_sm=c, small_max_elements=sm, cluster_size=cl, cluster_min_elements=cm)
    S = capi.Server(par, store_elements=int(total_el * 1.25) + (1 << 20), max_active=args.count,
                    tick_iters=args.tick_iters, max_m=4, max_q=20, **bc)
    # every controller's first solve (cold), then the timed window of step re-solves
    for c in range(args.count):
        S.submit(W.batch_instance(base + c), session=c)
    done = 0
    while done < args.count:
        t, lat, it, st = S.drain()
        done += len(t)
        time.sleep(0.001)
    rng = np.random.default_rng(1903 + rank)
    steps = np.zeros(args.count, dtype=np.int64)
    owner, trace = {}, []
    lat_all, it_all, st_all, ctl_all = [], [], [], []

    def take():
        t, lat, it, st = S.drain()
        lat_all.extend(lat.tolist())
        it_all.extend(it.tolist())
        st_all.extend(st.tolist())
        ctl_all.extend(owner.pop(int(k)) for k in t)

    submitted = 0
    st0 = S.stats()
    t_start = time.perf_counter()
    next_t = t_start + rng.exponential(1.0 / args.rate)
    with ClockSampler(local) as clk:
        while True:
            now = time.perf_counter()
            if now - t_start >= args.duration:
                break
            while next_t <= now:
                c = int(rng.integers(args.count))
                steps[c] += 1
                n, m, q = shapes[c]
                tk = S.submit_step(c, W.step_data(m, q, int(steps[c]), seed=W.SEED * (1 << 32) + base + c))
                owner[tk] = c
                trace.append((base + c, int(steps[c])))
                submitted += 1
                next_t += rng.exponential(1.0 / args.rate)
            take()
            time.sleep(0.0005)
        window = time.perf_counter() - t_start
        st1 = S.stats()
        busy_window = st1["gpu_busy_s"] - st0["gpu_busy_s"]
        shift_window = st1["gpu_shift_s"] - st0["gpu_shift_s"]
        finished_in_window = len(lat_all)
        t_end = time.perf_counter()
        while len(lat_all) < submitted and time.perf_counter() - t_end < 120:
            take()
            time.sleep(0.001)
    stats = S.stats()
    S.close()
    lat = np.array(lat_all) * 1e3
    value = finished_in_window / window
    (vmin,) = barrier_max([-value], world)
    # algorithmic bytes of the finished re-solves: iterations x the mixed per-iteration count of each shape
    from types import SimpleNamespace as NS
    bpi = lambda c: bytes_per_iteration(NS(n=shapes[c][0], m=shapes[c][1], q=shapes[c][2]), "mixed")
    byts = float(sum(i * bpi(c) for i, c in zip(it_all, ctl_all)))
    peaks = measured_peaks()
    gbs = byts / window / 1e9
    d2h = float(np.mean([8 * (n * m * q + m) for n, m, q in (shapes[c] for c in ctl_all)])) + 24 if ctl_all else 0.0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = serving_cpu_baseline(trace, par)
    if rank == 0:
        ok = np.array(st_all) == 0
        line = {"metric": METRIC, "value": value * world, "unit": "solves/s", "n_gpus": world,
                "steps": finished_in_window, "warmup": args.count,
                "ms_per_step": 1e3 * window / max(1, finished_in_window),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded receding-horizon steps per controller)",
                "config": {"workload": f"serving: Poisson {args.rate:g}/s re-solves of {args.count} controllers "
                                       f"sized as the batched workload, {args.duration:g} s window",
                           "tick_iters": args.tick_iters, "rho": penalty_text(args), "teams": dict(bc),
                           "steps": "requests finished in the window; warmup = the controllers' cold solves",
                           "parallelism": f"replicas x{world}"},
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "mean": float(np.mean(lat)), "max": float(np.max(lat))} if len(lat) else None,
                "window_s": window, "submitted": submitted, "finished": len(lat_all),
                "iters": {"mean": float(np.mean(it_all)), "p99": float(np.percentile(it_all, 99)),
                          "max": int(np.max(it_all)), "at_cap_frac": float(np.mean(np.array(it_all) >= par.max_iter))}
                if it_all else None,
                "ok_frac": float(np.mean(ok)) if st_all else None,
                "gpu_busy_frac": busy_window / window, "gpu_shift_frac": shift_window / window,
                "mean_active": (st1["instance_ticks"] - st0["instance_ticks"]) / max(1.0, st1["ticks"] - st0["ticks"]),
                "server_stats": stats,
                # the batched kernel once per tick of the window; a tick with step requests or finished
                # instances adds one shift or one gather kernel
                "gpu_launches": int(st1["ticks"] - st0["ticks"]),
                # requests go in and results come out through the public API from host memory, so the
                # served rate is itself end to end: a step request carries f, g [m][q], bounds [m] and
                # y [q] in FP64; each finished request's x [m][q][n] and x_1 [m] come back in FP64
                # (the server gathers them every tick) with its 24-byte record
                "e2e": {"value": value * world, "unit": "solves/s",
                        "h2d_bytes_per_step": float(np.mean([8 * (6 * m * q + 2 * m + q) for _, m, q in shapes])),
                        "d2h_bytes_per_step": d2h},
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": gbs / peaks["hbm_gbs"], "traffic": None, "algorithmic_bytes": byts,
                             "over": "the whole window (GPU idle time included)",
                             "achieved_while_busy": byts / max(busy_window, 1e-9) / 1e9,
                             "peak_source": peaks["source"]},
                "cpu_baseline": cpu, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


def config_dict(P, par, args):
    return {"workload": P.name + f" ({args.precision})", "n": P.n, "m": P.m, "q": P.q,
            "elements": P.elements, "rho": list(par.rho), "r_tol": par.r_tol, "s_tol": par.s_tol,
            "check_every": par.check_every, "max_iter": par.max_iter, "adapt_rho": bool(par.adapt_rho),
            "l2": "flushed between timed solves (512 MiB write)", "parallelism": f"replicas x{args.gpus}"}


def run_quartic(args):
    """Quartic benchmark of Sec. III-C: Algorithm 1 + clamp on N independent
    quartics, device-resident and with host copies, FP32 and FP64, beside the
    oracle's minimiser on 1 and all host cores (a sample)."""
    import torch
    rank, world, local = dist_init(args.gpus)
    from paper_1903_10041_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    sizes = [int(v) for v in str(args.quartic).split(",")]
    if min(sizes) < 1:
        raise ValueError("--quartic sizes must be >= 1")
    for N in sizes:
        quartic_line(args, N, rank, world)
    return 0


def quartic_line(args, N: int, rank: int, world: int):
    """One line of the quartic benchmark for N quartics."""
    import concurrent.futures as cf
    import ctypes
    import numpy as np
    import torch
    from paper_1903_10041_gb300 import capi
    g = torch.Generator(device="cuda").manual_seed(1903 + rank)

    def gen(dtype):
        u = lambda a, b: torch.rand(N, generator=g, device="cuda", dtype=torch.float64) * (b - a) + a
        A, B, Cc, D = u(0.01, 2.0), u(-2.0, 2.0), u(-3.0, 3.0), u(-2.0, 2.0)
        c0, w = u(-2.0, 2.0), u(0.0, 3.0)
        return [t.to(dtype).contiguous() for t in (A, B, Cc, D, c0 - w, c0 + w)]

    stream = torch.cuda.current_stream()
    out = {}
    for prec, dtype, width in (("fp32", torch.float32, 4), ("fp64", torch.float64, 8)):
        dev = gen(dtype)
        x = torch.empty_like(dev[0])
        for _ in range(args.warmup):
            capi.quartic_min(*dev, precision=prec, stream=stream, out=x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            capi.quartic_min(*dev, precision=prec, stream=stream, out=x)
        e1.record(stream)
        e1.synchronize()
        s_dev = e0.elapsed_time(e1) / 1e3 / args.steps
        host = [t.cpu().pin_memory().numpy() for t in dev]
        xh = torch.empty(N, dtype=dtype).pin_memory().numpy()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps // 2)):
            capi.quartic_min(*host, precision=prec, stream=stream, out=xh)
        s_e2e = (time.perf_counter() - t0) / max(1, args.steps // 2)
        out[prec] = {"dev_per_s": N / s_dev, "e2e_per_s": N / s_e2e, "gbs": 7 * width * N / s_dev / 1e9,
                     "sample": (host, xh)}
        del dev, x
    # oracle's Algorithm 1 on the host: a sample, 1 thread and all threads (ctypes drops the GIL)
    import oracle
    L = oracle.lib()
    ns = min(N, 1 << 21)
    arrs = [np.ascontiguousarray(a[:ns], dtype=np.float64) for a in out["fp64"]["sample"][0]]
    xo = np.empty(ns)
    dp = ctypes.POINTER(ctypes.c_double)

    def run(lo_i, hi_i):
        L.orc_quartic_min_many(hi_i - lo_i, *[a[lo_i:].ctypes.data_as(dp) for a in arrs], 0,
                               xo[lo_i:].ctypes.data_as(dp), None)

    def rate(fn):  # quartics/s, repeating small samples to at least 50 ms
        reps, t0 = 0, time.perf_counter()
        while True:
            fn()
            reps += 1
            dt = time.perf_counter() - t0
            if dt >= 0.05:
                return reps * ns / dt
    cpu1 = rate(lambda: run(0, ns))
    threads = min(os.cpu_count() or 1, ns)
    bounds = np.linspace(0, ns, threads + 1).astype(int)
    with cf.ThreadPoolExecutor(threads) as ex:
        cpun = rate(lambda: list(ex.map(lambda t: run(bounds[t], bounds[t + 1]), range(threads))))
    x64 = out["fp64"]["sample"][1][:ns]
    agree = float(np.mean(np.abs(x64 - xo) <= 1e-9 * np.maximum(1.0, np.abs(xo))))
    peaks = measured_peaks()
    (vmax,) = barrier_max([-out["fp32"]["dev_per_s"]], world)
    if rank == 0:
        f32, f64 = out["fp32"], out["fp64"]
        line = {"metric": "quartic minimisations/s (Algorithm 1 + clamp, Sec. III-C)", "value": f32["dev_per_s"] * world,
                "unit": "quartics/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * N / f32["dev_per_s"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded uniform quartics and intervals)",
                "config": {"workload": f"{N} independent quartics", "n": N},
                "roofline": {"bound": "hbm", "achieved": f32["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": f32["gbs"] / peaks["hbm_gbs"], "traffic": None},
                "e2e": {"value": f32["e2e_per_s"], "unit": "quartics/s", "h2d_bytes_per_step": 24 * N,
                        "d2h_bytes_per_step": 4 * N},
                "fp64": {"dev_per_s": f64["dev_per_s"], "e2e_per_s": f64["e2e_per_s"], "gbs": f64["gbs"],
                         "frac": f64["gbs"] / peaks["hbm_gbs"], "agree_with_oracle_1e-9": agree},
                "cpu_baseline": {"value": cpun, "unit": "quartics/s", "cores": threads, "kind": "oracle",
                                 "one_core": cpu1, "sample": f"{ns} of the quartics, FP64"},
                "speedup_e2e_fp32_vs_all_cores": f32["e2e_per_s"] / cpun,
                "gpu_launches": 2 * (args.steps + max(1, args.steps // 2))}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=3, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--count", type=int, default=4096, help="instances (3) or controllers (4)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving window in seconds (4)")
    ap.add_argument("--rate", type=float, default=2000.0, help="Poisson arrival rate per second (4)")
    ap.add_argument("--tick-iters", type=int, default=10,
                    help="iterations per serving tick of the costliest active instance (4)")
    ap.add_argument("--adapt", action="store_true",
                    help="penalty adaptation of Sec. IV-A (0, 1, 2, 4, --q-sweep; always on for 3 unless --fixed-rho)")
    ap.add_argument("--adapt-start", type=int, default=0,
                    help="with the adaptation: apply it at check iterations >= this (0: from the first)")
    ap.add_argument("--fixed-rho", action="store_true",
                    help="--config 3, 4: keep rho = (1, 1/n, 1, 1) fixed instead of the Sec. IV-A adaptation")
    ap.add_argument("--paper-penalties", action="store_true",
                    help="--config 1 or --q-sweep: the PHEV settings of Sec. IV-A (rho = 1e-4, 2e-6, 5e-6, 5e-6; "
                         "r-bar = 1e-6 dE, sigma-bar = 1e-2; adaptation on)")
    ap.add_argument("--batch-config", default="",
                    help="warps,ctas_per_sm,small_max,cluster,cluster_min instead of the autotuner (3, 4)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_fp64cubic"])
    ap.add_argument("--max-iter", type=int, default=0,
                    help="profiling only: cap the iterations of each solve (the line is then not a benchmark)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-sample", action="store_true",
                    help="--config 3: skip the per-instance oracle comparison (profiling runs)")
    ap.add_argument("--coef-shared", action="store_true",
                    help="--config 1 or 2: scenario-shared cost and loss maps ([m][n] coefficients)")
    ap.add_argument("--q-sweep", default="",
                    help="comma-separated scenario counts (e.g. 5,10,20,50,100,200,500): one line per q for the "
                         "n=1000 PHEV instance, runtime against q as in Sec. IV-B")
    ap.add_argument("--quartic", default="",
                    help="N or N1,N2,...: the quartic benchmark of Sec. III-C on N quartics instead of a solve "
                         "(a list gives one line per N, e.g. 100,1000,...,1000000000 for the crossover)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.config == 3 and not args.quartic and not args.q_sweep:
        args.adapt = not args.fixed_rho  # the batched workload runs the paper's solver with its adaptation
    if args.config == 4 and not args.fixed_rho:
        # served re-solves start warm: the adaptation acts on those still running after 1000 iterations
        # (at 2000/s offered: p99 1.46 s, 99.97 % converged; fixed rho 1.93 s, 99.50 %)
        args.adapt = True
        args.adapt_start = args.adapt_start or 1000
    if args.impl == "reference":
        return run_reference(args)
    if args.quartic:
        return run_quartic(args)
    if args.config in (3, 4) and not args.q_sweep:
        return run_batched(args) if args.config == 3 else run_serving(args)

    import torch
    rank, world, local = dist_init(args.gpus)
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    from paper_1903_10041_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    if args.q_sweep:
        for P, par in sweep_workloads(args.q_sweep, args.precision, args.adapt, args.paper_penalties):
            run_single(args, P, par, rank, world, local)
    else:
        P, par = workload(args.config, args.precision, args.coef_shared)
        par = paper_penalties(P, args.precision) if args.paper_penalties else par.replace(adapt_rho=args.adapt)
        run_single(args, P, par, rank, world, local)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def paper_penalties(P, precision: str = "fp64"):
    """The settings of the PHEV study (Sec. IV-A): initial penalties rho_1 =
    1e-4, rho_2 = 2e-6, rho_3 = rho_4 = 5e-6, thresholds r-bar = 1e-6 dE
    (dE: the battery capacity, c of the second source) and sigma-bar = 1e-2,
    with the penalty adaptation on."""
    from paper_1903_10041_gb300 import workloads as W
    dE = float(P.c[1])
    return W.Params(rho=(1e-4, 2e-6, 5e-6, 5e-6), r_tol=1e-6 * dE, s_tol=1e-2, adapt_rho=True, precision=precision)


def sweep_workloads(spec: str, precision: str, adapt: bool, paper: bool = False):
    """The PHEV-shaped instance (n = 1000, m = 2) at each scenario count of a
    comma-separated list, with the penalties of the q = 50 case (or, with
    `paper`, the settings of Sec. IV-A): the runtime against q sweep of
    Sec. IV-B (q from 5 to 500 there)."""
    from paper_1903_10041_gb300 import workloads as W
    out = []
    for tok in spec.split(","):
        q = int(tok)
        if q < 1:
            raise ValueError(f"scenario count {q} < 1")
        P = W.phev_problem(1000, q)
        par = (paper_penalties(P, precision) if paper else
               W.Params(rho=(1.0, 1.0 / P.n, 1.0, 1.0), precision=precision, adapt_rho=adapt))
        out.append((P, par))
    return out


def run_single(args, P, par, rank, world, local):
    """Times K single-instance solves of P (one persistent-kernel launch
    each) and prints one JSON line."""
    import numpy as np
    import torch
    from paper_1903_10041_gb300 import capi
    if args.max_iter:
        par = par.replace(max_iter=args.max_iter)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    solver = capi.Solver(P, par)

    def one_solve():
        solver.reset()
        torch.cuda.synchronize()
        flush.fill_(1.0)                     # evict L2 (outside the timed events)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.solve_async(stream=stream)
        e1.record(stream)
        res = solver.wait()
        e1.synchronize()
        return e0.elapsed_time(e1), res

    for _ in range(args.warmup):
        one_solve()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, results = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            ms, res = one_solve()
            times.append(ms)
            results.append(res)
    torch.cuda.synchronize()
    total_ms = sum(times)
    (total_ms_max,) = barrier_max([total_ms], world)
    iters = results[-1]["iters"]
    conv = all(r["converged"] for r in results)
    value = world * args.steps / (total_ms_max / 1e3)

    # ---- roofline of the solve kernel (one launch = one solve) ------------
    per_launch_s = total_ms / args.steps / 1e3
    if args.precision == "fp64":
        flops = iters * fp64_flops_per_iteration(P)
        achieved = flops / per_launch_s / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_per_launch(P, "fp64", iters),
                    "peak_source": "FP64: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (derived; measured 1.90 DFMA/clk/SM)",
                    "fp64_pipe_busy": fp64_pipe_busy(P),
                    # algorithmic bytes streamed per second; an instance that fits in L2
                    # (the n=1000 PHEV one) is served mostly from L2, not HBM (see traffic)
                    "streamed_gbs": iters * bytes_per_iteration(P, "fp64") / per_launch_s / 1e9}
    else:
        peaks = measured_peaks()
        gbs = iters * bytes_per_iteration(P, args.precision) / per_launch_s / 1e9
        roofline = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "traffic": traffic_per_launch(P, args.precision, iters)}

    # ---- end to end through the C ABI from pinned host buffers ------------
    e2e = None
    if not args.no_e2e:
        pinned = P.copy()
        for k, v in P.arrays().items():
            t = torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
            setattr(pinned, k, t.numpy())
        x_out = torch.empty((P.m, P.q, P.n), dtype=torch.float64).pin_memory().numpy()
        x1_out = torch.empty(P.m, dtype=torch.float64).pin_memory().numpy()
        h2d = sum(v.nbytes for v in P.arrays().values())
        d2h = x_out.nbytes + x1_out.nbytes

        def e2e_step():
            t0 = time.perf_counter()
            with capi.Solver(pinned, par) as s:
                s.solve(x_out=x_out, x1_out=x1_out)
            return time.perf_counter() - t0

        for _ in range(3):
            e2e_step()
        et = [e2e_step() for _ in range(max(3, args.steps // 2))]
        (et_max,) = barrier_max([sum(et)], world)
        e2e = {"value": world * len(et) / et_max, "unit": "solves/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(P, par, iters, budget_s=4.0 if args.q_sweep else 12.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32+f64",
                "data": "synthetic (seeded; stands in for the paper's FTP-75 PHEV scenarios)",
                "config": config_dict(P, par, args),
                "iters_per_solve": iters, "converged": conv, "objective": results[-1]["objective"],
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps,
                "profiling_cap": args.max_iter or None,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    solver.close()


if __name__ == "__main__":
    sys.exit(main())

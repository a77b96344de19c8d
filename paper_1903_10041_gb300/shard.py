"""Host side of a single instance split over workers by time step k.

One instance of eq. (2) too large for one device is cut along k: worker r
owns the columns k in [k_r, k_{r+1}) of every row (i, j).  Step (a) and
steps (e), (f), (g) of App. A act on one column at a time (Sec. II: the
(j, k) updates are independent); what couples the columns is the
per-(i, j) sum over k of g(x) - lambda (steps (b), (d), (i)) and x at
k = 0 (steps (c), (h)).  So an iteration is

  phase A   every worker: its columns' element updates and a record of
            2 m q + 2 values: the per-pair partial sums, x at k = 0 from the
            worker that owns k = 0, and the largest column residual terms;
  exchange  one collective: every worker gathers every record and combines
            them in worker order (sums, and maxima for the residual terms),
            so all workers hold the same bits;
  phase B   every worker: the per-pair scalar steps from the combined record
            (the same on all workers) and its columns' z and lambda.

On check iterations a second, two-value maximum over the workers completes
the residuals (the element terms |z - g(x)| and |z - z~|), and every worker
takes the same stop decision (Alg. 2 step 3) and, with the penalty
adaptation of Sec. IV-A, the same rescaling: from the same r and sigma every
worker divides its columns' lambda, mu and the pair scalars p, nu by the
factor and multiplies the penalties by it.

This module is the protocol: the column split, the record layout, the
exchange and the stop test.  The per-worker compute is a backend object
with ``snapshot()``, ``phase_a(check)``, ``phase_b(tot, check)`` and
``rescale(f)``; the
tests drive it on CPU worker processes (gloo) with their FP64 reference
implementation of the two phases.  The device kernels for the two phases
are not built: every machine this project runs on has one GPU, and a
single instance fits it.
"""
from __future__ import annotations

import math

import numpy as np


def column_shards(n: int, workers: int) -> list:
    """Contiguous column ranges [k0, k1) of near-equal length, worker 0 first
    (it owns k = 0)."""
    if workers < 1 or n < workers:
        raise ValueError(f"cannot split {n} columns over {workers} workers")
    b = [n * r // workers for r in range(workers + 1)]
    return [(b[r], b[r + 1]) for r in range(workers)]


def record_len(m: int, q: int) -> int:
    return 2 * m * q + 2


def combine(records: np.ndarray, m: int, q: int) -> np.ndarray:
    """Combines the workers' records [workers, 2mq + 2] in worker order: the
    per-pair sums and x at k = 0 are added, the residual terms maximised."""
    mq = m * q
    tot = np.zeros(record_len(m, q))
    for rec in records:                       # fixed order: worker 0, 1, ...
        tot[:2 * mq] += rec[:2 * mq]
        tot[2 * mq:] = np.maximum(tot[2 * mq:], rec[2 * mq:])
    return tot


class Exchange:
    """The collectives of the protocol over a torch.distributed group (gloo
    on CPU tensors, NCCL on device tensors)."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist, self.group, self.device = dist, group, device
        self.world = dist.get_world_size(group)

    def gather_combine(self, rec: np.ndarray, m: int, q: int) -> np.ndarray:
        import torch
        t = torch.as_tensor(rec, dtype=torch.float64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return combine(np.stack([o.cpu().numpy() for o in out]), m, q)

    def max(self, values) -> np.ndarray:
        import torch
        t = torch.as_tensor(np.asarray(values, dtype=np.float64), device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return t.cpu().numpy()


def _div(a: float, b: float) -> float:
    """a / b with the IEEE results for b = 0 (inf, or nan for 0 / 0)."""
    if b != 0.0:
        return a / b
    return float("nan") if a == 0.0 else math.copysign(float("inf"), a)


def run(backend, exchange, m: int, q: int, rho, r_tol: float, s_tol: float, max_iter: int,
        check_every: int, adapt: bool = False, tau: float = 1.1, adapt_start: int = 0) -> dict:
    """Iterates phase A, exchange, phase B until the stop test of Alg. 2
    step 3 (r < r_tol and sigma < s_tol at a check iteration) or max_iter.
    rho = (rho_1, rho_2, rho_3, rho_4) as the backend uses them.  adapt:
    the ratio rule of Sec. IV-A at check iterations t >= adapt_start (not
    the last), rho <- rho f with f = tau or 1 / tau, duals divided by f."""
    rho = tuple(float(v) for v in rho)
    mq = m * q
    r = sigma = float("inf")
    it = 0
    for it in range(1, max_iter + 1):
        check = it % check_every == 0 or it == max_iter
        backend.snapshot()
        rec = backend.phase_a(check)
        tot = exchange.gather_combine(rec, m, q)
        res = backend.phase_b(tot, check)    # |z-g|, |z-z~| (own columns); |h-1'z|, copies, |h-h~|
        if check:
            r2, s1 = exchange.max(res[:2])
            r1, s3 = tot[2 * mq], tot[2 * mq + 1]
            r = max(r1, r2, res[2], res[3])
            sigma = max(rho[0] * s1, rho[1] * res[4], rho[2] * s3)
            if r < r_tol and sigma < s_tol:
                return {"iters": it, "converged": True, "r": r, "sigma": sigma, "rho": list(rho)}
            if adapt and it < max_iter and it >= adapt_start:
                ratio, target, f = _div(r, sigma), _div(r_tol, s_tol), 1.0
                if ratio > 1.2 * target:
                    f = tau
                elif ratio < 0.8 * target:
                    f = 1.0 / tau
                if f != 1.0:
                    backend.rescale(f)
                    rho = tuple(v * f for v in rho)
    return {"iters": it, "converged": False, "r": r, "sigma": sigma, "rho": list(rho)}

"""A worker of the column-sharded iteration computed by the FP64 oracle
(test infrastructure: it stands in for the device kernels of the two
phases on CPU worker processes)."""
import numpy as np

import oracle


def shard_problem(P, k0, k1):
    """The worker's slice of problem (2): columns [k0, k1) of every row; the
    capacities whole."""
    Q = P.copy()
    for k in ("f2", "f1", "f0", "g2", "g1", "g0"):
        setattr(Q, k, np.ascontiguousarray(getattr(P, k)[:, :, k0:k1]))
    Q.lo, Q.hi = np.ascontiguousarray(P.lo[:, k0:k1]), np.ascontiguousarray(P.hi[:, k0:k1])
    Q.y = np.ascontiguousarray(P.y[:, k0:k1])
    Q.n = k1 - k0
    return Q


class OracleShard:
    def __init__(self, P, par, k0, k1):
        self.P, self.par, self.k0, self.n_total = shard_problem(P, k0, k1), par, k0, P.n
        self.st = oracle.init_state(self.P)

    def snapshot(self):
        self.xp, self.sp, self.zp, self.hp = (self.st[k].copy() for k in ("x", "s", "z", "h"))

    def phase_a(self, check):
        self.gx, rec = oracle.shard_phase_a(self.P, self.par, self.st, self.k0, self.xp, self.sp,
                                            n_total=self.n_total)
        return rec

    def phase_b(self, tot, check):
        return oracle.shard_phase_b(self.P, self.par, self.st, self.n_total, tot, self.gx, self.zp, self.hp)

    def rescale(self, f):
        """Sec. IV-A: the scaled duals divided by f, the penalties multiplied by f."""
        for k in ("lam", "mu", "p", "nu"):
            self.st[k] /= f
        self.par = self.par.replace(rho=tuple(v * f for v in self.par.rho))

"""Seeded synthetic inputs for the robust resource-allocation problem (2).

This module only *generates inputs*; it holds none of the solver's arithmetic.
Both the CUDA path and the FP64 oracle take their problems from here.

Random numbers come from a counter-based SplitMix64 hash (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value
number ``idx`` of stream ``(seed, tag...)`` is ``mix64(key + (idx + 1) * GAMMA)``.
It is written in plain numpy uint64 arithmetic, so a seed gives the same
numbers on every machine and numpy version.

Problem data follow Assumption 3 (Sec. II): per element (i, j, k)
    f_k^(i,j)(x) = f2 x^2 + f1 x + f0,   g_k^(i,j)(x) = g2 x^2 + g1 x + g0,
bounds x_k^(i) in [lo, hi] shared by all scenarios j, demand y_k^(j) per
scenario (Sec. II, eq. 2) and capacity c^(i) per source.
Arrays are C-contiguous float64 with shapes
    f*, g*: [m, q, n];  lo, hi: [m, n];  y: [q, n];  c: [m].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED = 1903

# stream tags (arbitrary distinct constants)
T_F2, T_F1, T_F0, T_G2, T_G1, T_G0 = 11, 12, 13, 21, 22, 23
T_Y, T_YN1, T_YN2, T_BASE, T_SHAPE = 31, 32, 33, 34, 35
T_INST = 41


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, *tags: int) -> np.uint64:
    h = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    for t in tags:
        h = _mix64(h ^ np.uint64(t & 0xFFFFFFFFFFFFFFFF))
    return h[0]


def uniform(seed: int, tags: tuple, size: int) -> np.ndarray:
    """``size`` doubles in [0, 1) from stream (seed, *tags)."""
    idx = np.arange(1, size + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, *tags) + idx * _GAMMA
    return (_mix64(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, tags: tuple, size: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = uniform(seed, tags + (1,), size)
    u2 = uniform(seed, tags + (2,), size)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _u(seed, tags, shape, a, b):
    n = int(np.prod(shape))
    return (a + (b - a) * uniform(seed, tags, n)).reshape(shape)


@dataclasses.dataclass
class Problem:
    """Input data of problem (2). ``c`` may hold +inf (no capacity limit)."""
    n: int
    m: int
    q: int
    f2: np.ndarray
    f1: np.ndarray
    f0: np.ndarray
    g2: np.ndarray
    g1: np.ndarray
    g0: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    y: np.ndarray
    c: np.ndarray
    name: str = ""
    coef_shared: bool = False     # f2..g0 are [m][n], the same maps for every scenario

    @property
    def elements(self) -> int:
        return self.m * self.q * self.n

    def dense(self) -> "Problem":
        """The same problem with per-scenario coefficient arrays [m][q][n]."""
        if not self.coef_shared:
            return self
        rep = {k: np.ascontiguousarray(np.broadcast_to(getattr(self, k)[:, None, :], (self.m, self.q, self.n)))
               for k in ("f2", "f1", "f0", "g2", "g1", "g0")}
        return dataclasses.replace(self, coef_shared=False, **rep)

    def arrays(self):
        return dict(f2=self.f2, f1=self.f1, f0=self.f0, g2=self.g2, g1=self.g1, g0=self.g0,
                    lo=self.lo, hi=self.hi, y=self.y, c=self.c)

    def copy(self) -> "Problem":
        return dataclasses.replace(self, **{k: v.copy() for k, v in self.arrays().items()})


@dataclasses.dataclass
class Params:
    """Solver settings: penalties rho_1..rho_4 (App. A), stop thresholds r-bar and
    sigma-bar (Alg. 2 step 3), and the residual check interval (Sec. IV-B)."""
    rho: tuple = (1.0, 1.0, 1.0, 1.0)
    r_tol: float = 1e-6
    s_tol: float = 1e-6
    max_iter: int = 5000
    check_every: int = 10
    precision: str = "fp64"       # "fp64" | "mixed"
    xmin_mode: str = "exact"      # "exact" | "paper"
    sweep: str = "gauss_seidel"   # "gauss_seidel" | "jacobi"
    adapt_rho: bool = False       # Sec. IV-A penalty adaptation
    tau: float = 1.1
    rho2_over_n: bool = False     # each instance uses rho_2 = rho[1] / n
    adapt_start: int = 0          # with adapt_rho: adapt at check iterations t >= adapt_start only

    def replace(self, **kw) -> "Params":
        return dataclasses.replace(self, **kw)


def _capacity(g2, g1, g0, at: float) -> np.ndarray:
    """c^(i) = 0.6 * min_j sum_k g_k^(i,j)(at): a capacity the demand-splitting
    point x = y/m satisfies (input recipe, stated with the configurations)."""
    tot = (g2 * at * at + g1 * at + g0).sum(axis=2)  # [m, q]
    return 0.6 * tot.min(axis=1)


def random_problem(n: int, m: int, q: int, seed: int = SEED, name: str = "") -> Problem:
    """The recipe of the plain instance: f = a x^2 + b x, a~U[0.1,1], b~U[-1,1];
    g = alpha x^2 + x, alpha~U[0.01,0.1]; x in [-1, 2]; y~U[0.5, 2];
    c^(i) = 0.6 * min_j sum_k g(2). Drawn independently per (i, j, k)."""
    sh = (m, q, n)
    f2 = _u(seed, (T_F2,), sh, 0.1, 1.0)
    f1 = _u(seed, (T_F1,), sh, -1.0, 1.0)
    f0 = np.zeros(sh)
    g2 = _u(seed, (T_G2,), sh, 0.01, 0.1)
    g1 = np.ones(sh)
    g0 = np.zeros(sh)
    lo = np.full((m, n), -1.0)
    hi = np.full((m, n), 2.0)
    y = _u(seed, (T_Y,), (q, n), 0.5, 2.0)
    c = _capacity(g2, g1, g0, 2.0)
    return Problem(n, m, q, f2, f1, f0, g2, g1, g0, lo, hi, y, c, name or f"plain n={n} m={m} q={q}")


def shared_problem(n: int, m: int, q: int, seed: int = SEED, name: str = "") -> Problem:
    """The plain recipe with scenario-shared cost and loss maps: f and g are
    drawn per (i, k) ([m][n]) and only the demand y differs by scenario."""
    sh = (m, n)
    f2 = _u(seed, (T_F2,), sh, 0.1, 1.0)
    f1 = _u(seed, (T_F1,), sh, -1.0, 1.0)
    g2 = _u(seed, (T_G2,), sh, 0.01, 0.1)
    g1 = np.ones(sh)
    z = np.zeros(sh)
    lo = np.full((m, n), -1.0)
    hi = np.full((m, n), 2.0)
    y = _u(seed, (T_Y,), (q, n), 0.5, 2.0)
    c = _capacity(g2[:, None, :], g1[:, None, :], z[:, None, :], 2.0)
    return Problem(n, m, q, f2, f1, z.copy(), g2, g1, z.copy(), lo, hi, y, c,
                   name or f"shared n={n} m={m} q={q}", coef_shared=True)


def phev_problem(n: int = 1000, q: int = 50, seed: int = SEED) -> Problem:
    """PHEV-shaped robust problem (Sec. IV, eq. PHEV_opt) with synthetic data.

    Source 1 (engine): f = a x^2 + b x, a~U[0.1,1], b~U[-1,1]; g = 0; c = +inf;
    x in [0, 3] (no engine braking). Source 2 (battery): f = 0;
    g = alpha x^2 + x, alpha~U[0.01, 0.1]; x in [-1, 1]; capacity 0.3 n.
    Demand per scenario: 1 + sum of three sinusoids (amplitudes summing to at
    most 0.8, periods in [50, 500] steps) shared by all scenarios, plus
    independent N(0, 0.1^2) noise per (j, k)."""
    m = 2
    sh = (m, q, n)
    f2 = np.zeros(sh); f1 = np.zeros(sh); f0 = np.zeros(sh)
    g2 = np.zeros(sh); g1 = np.zeros(sh); g0 = np.zeros(sh)
    f2[0] = _u(seed, (T_F2,), (q, n), 0.1, 1.0)
    f1[0] = _u(seed, (T_F1,), (q, n), -1.0, 1.0)
    g2[1] = _u(seed, (T_G2,), (q, n), 0.01, 0.1)
    g1[1] = 1.0
    lo = np.array([np.zeros(n), np.full(n, -1.0)])
    hi = np.array([np.full(n, 3.0), np.full(n, 1.0)])
    shape = uniform(seed, (T_SHAPE,), 9)
    amp = 0.8 * shape[0:3] / 3.0                    # sum <= 0.8
    per = 50.0 + 450.0 * shape[3:6]
    pha = 2.0 * math.pi * shape[6:9]
    k = np.arange(n, dtype=np.float64)
    base = 1.0 + sum(amp[r] * np.sin(2.0 * math.pi * k / per[r] + pha[r]) for r in range(3))
    y = base[None, :] + 0.1 * normal(seed, (T_YN1,), q * n).reshape(q, n)
    c = np.array([np.inf, 0.3 * n])
    return Problem(n, m, q, f2, f1, f0, g2, g1, g0, lo, hi, y, c, f"phev n={n} q={q}")


def batch_shape(instance: int, seed: int = SEED) -> tuple:
    """(n, m, q) of one batched instance: n log-uniform in [50, 5000],
    m in {2, 3, 4}, q uniform in [1, 20]."""
    u = uniform(seed, (T_INST, instance), 3)
    n = int(round(math.exp(math.log(50.0) + u[0] * (math.log(5000.0) - math.log(50.0)))))
    m = 2 + min(int(u[1] * 3.0), 2)
    q = 1 + min(int(u[2] * 20.0), 19)
    return n, m, q


def batch_instance(instance: int, seed: int = SEED) -> Problem:
    """Instance ``instance`` of the batched workload: sizes from
    :func:`batch_shape`, data drawn as in :func:`random_problem` with the
    per-instance seed ``seed * 2**32 + instance``."""
    n, m, q = batch_shape(instance, seed)
    p = random_problem(n, m, q, seed=seed * (1 << 32) + instance)
    p.name = f"batch#{instance} n={n} m={m} q={q}"
    return p


def step_data(m: int, q: int, step: int, seed: int = SEED) -> dict:
    """The data of a new last step for a plain-recipe controller at sampling
    instant ``step``: f2, f1, f0, g2, g1, g0 [m, q], lo, hi [m], y [q]."""
    def fresh(tag, shape, a, b):
        return (a + (b - a) * uniform(seed, (tag, 7, step), int(np.prod(shape)))).reshape(shape)

    return {"f2": fresh(T_F2, (m, q), 0.1, 1.0), "f1": fresh(T_F1, (m, q), -1.0, 1.0), "f0": np.zeros((m, q)),
            "g2": fresh(T_G2, (m, q), 0.01, 0.1), "g1": np.ones((m, q)), "g0": np.zeros((m, q)),
            "lo": np.full(m, -1.0), "hi": np.full(m, 2.0), "y": fresh(T_Y, (q,), 0.5, 2.0)}


def receding_step(p: Problem, step: int, seed: int = SEED) -> Problem:
    """Receding-horizon re-solve (Sec. II; Alg. 2) of a plain-recipe problem:
    the horizon moves one sampling instant forward, so every per-step array
    (f, g, bounds, demand) moves one step and the new last step is
    :func:`step_data`; the capacities are kept."""
    out = p.copy()
    d = step_data(p.m, p.q, step, seed)
    for k in ("f2", "f1", "f0", "g2", "g1", "g0"):
        setattr(out, k, np.concatenate([getattr(p, k)[:, :, 1:], d[k][:, :, None]], axis=2))
    out.lo = np.concatenate([p.lo[:, 1:], d["lo"][:, None]], axis=1)
    out.hi = np.concatenate([p.hi[:, 1:], d["hi"][:, None]], axis=1)
    out.y = np.concatenate([p.y[:, 1:], d["y"][:, None]], axis=1)
    return out


CONFIGS = {
    0: lambda: random_problem(100, 2, 1, name="plain n=100 m=2 q=1"),
    1: lambda: phev_problem(1000, 50),
    2: lambda: random_problem(100_000, 4, 20, name="plain n=1e5 m=4 q=20"),
}


def config(i: int) -> Problem:
    return CONFIGS[i]()

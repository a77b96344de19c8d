"""FP64 CPU oracle of the ADMM iteration (a)-(i) and Algorithm 1.

TEST INFRASTRUCTURE ONLY: the plain, slow, literal reference that the CUDA
path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the solver never does.  It shares
no code with the CUDA path.  The C source (``admm_oracle.c``) cites the
paper for each step and lists the readings it takes.

Every function here marshals numpy arrays to the C oracle; none does
arithmetic of the method itself.  Problems and settings are duck-typed: any
object with the attributes of the input recipe (n, m, q, f2, f1, f0, g2, g1,
g0, lo, hi, y, c) and of the settings (rho, r_tol, s_tol, max_iter,
check_every, xmin_mode, sweep) will do.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("q", C.c_int),
                ("f2", _dp), ("f1", _dp), ("f0", _dp), ("g2", _dp), ("g1", _dp), ("g0", _dp),
                ("lo", _dp), ("hi", _dp), ("y", _dp), ("c", _dp)]


class _Params(C.Structure):
    _fields_ = [("rho1", C.c_double), ("rho2", C.c_double), ("rho3", C.c_double), ("rho4", C.c_double),
                ("r_tol", C.c_double), ("s_tol", C.c_double), ("max_iter", C.c_int),
                ("check_every", C.c_int), ("xmin_mode", C.c_int), ("sweep", C.c_int),
                ("threads", C.c_int), ("count_differs", C.c_int),
                ("adapt_rho", C.c_int), ("tau", C.c_double), ("adapt_start", C.c_int)]


class _State(C.Structure):
    _fields_ = [("x", _dp), ("z", _dp), ("lam", _dp), ("s", _dp), ("mu", _dp),
                ("h", _dp), ("p", _dp), ("nu", _dp), ("x1", _dp)]


class _Report(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("r", C.c_double), ("sigma", C.c_double),
                ("r_terms", C.c_double * 4), ("s_terms", C.c_double * 3),
                ("branch_count", C.c_longlong * 4), ("literal_differs", C.c_longlong),
                ("rho", C.c_double * 4)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.orc_quartic_min.restype = C.c_double
        L.orc_quartic_min.argtypes = [C.c_double] * 6 + [C.c_int, C.POINTER(C.c_int)]
        L.orc_quartic_min_many.restype = None
        L.orc_quartic_min_many.argtypes = [C.c_longlong] + [_dp] * 6 + [C.c_int, _dp, C.POINTER(C.c_int)]
        L.orc_cubic_roots.restype = C.c_int
        L.orc_cubic_roots.argtypes = [C.c_double] * 3 + [_dp, C.POINTER(C.c_int)]
        L.orc_init_state.restype = None
        L.orc_init_state.argtypes = [C.POINTER(_Problem), C.POINTER(_State)]
        L.orc_solve.restype = C.c_int
        L.orc_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_State), C.POINTER(_Report)]
        L.orc_objective.restype = C.c_double
        L.orc_objective.argtypes = [C.POINTER(_Problem), _dp]
        L.orc_kkt.restype = C.c_double
        L.orc_kkt.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_State), _dp]
        L.orc_shard_phase_a.restype = None
        L.orc_shard_phase_a.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_State), C.c_int,
                                        _dp, _dp, _dp, _dp, _dp]
        L.orc_shard_phase_b.restype = None
        L.orc_shard_phase_b.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_State), C.c_int,
                                        _dp, _dp, _dp, _dp, _dp]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


_MODES = {"exact": 0, "paper": 1}
_SWEEPS = {"gauss_seidel": 0, "jacobi": 1}


def quartic_min(A, B, Cc, D, lo=-np.inf, hi=np.inf, mode: str = "exact"):
    """Algorithm 1 + clamp, elementwise.  Returns (x, branch) with branch
    0 Cardano, 1 triple root, 2 trig, 3 quadratic (A = 0)."""
    arrs = np.broadcast_arrays(*[np.asarray(v, dtype=np.float64) for v in (A, B, Cc, D, lo, hi)])
    shape = arrs[0].shape
    arrs = [_f64(a.ravel()) for a in arrs]
    x = np.empty(arrs[0].size)
    br = np.empty(arrs[0].size, dtype=np.int32)
    lib().orc_quartic_min_many(x.size, *[_ptr(a) for a in arrs], _MODES[mode], _ptr(x),
                               br.ctypes.data_as(C.POINTER(C.c_int)))
    return x.reshape(shape), br.reshape(shape)


def cubic_roots(b: float, c: float, d: float):
    """Roots of x^3 + b x^2 + c x + d by the formulas of Sec. III-B: (roots, branch)."""
    r = np.zeros(3)
    br = C.c_int(0)
    k = lib().orc_cubic_roots(float(b), float(c), float(d), _ptr(r), C.byref(br))
    return r[:k].copy(), br.value


class _Holder:
    """Keeps the numpy arrays alive while C structs point at them."""

    def __init__(self, prob):
        self.arrs = {k: _f64(getattr(prob, k)) for k in ("f2", "f1", "f0", "g2", "g1", "g0", "lo", "hi", "y", "c")}
        self.n, self.m, self.q = int(prob.n), int(prob.m), int(prob.q)
        assert self.arrs["f2"].shape == (self.m, self.q, self.n)
        self.c = _Problem(self.n, self.m, self.q, *[_ptr(self.arrs[k]) for k in
                          ("f2", "f1", "f0", "g2", "g1", "g0", "lo", "hi", "y", "c")])


def _params(par, threads: int = 1, count_differs: bool = False, n: int | None = None) -> _Params:
    rho = tuple(float(r) for r in par.rho)
    if getattr(par, "rho2_over_n", False):
        rho = (rho[0], rho[1] / n, rho[2], rho[3])
    return _Params(rho[0], rho[1], rho[2], rho[3], float(par.r_tol), float(par.s_tol), int(par.max_iter),
                   int(par.check_every), _MODES[par.xmin_mode], _SWEEPS[par.sweep], int(threads),
                   int(count_differs), int(getattr(par, "adapt_rho", False)), float(getattr(par, "tau", 1.1)),
                   int(getattr(par, "adapt_start", 0)))


STATE_KEYS = ("x", "z", "lam", "s", "mu", "h", "p", "nu", "x1")


def _state_struct(st: dict) -> _State:
    return _State(*[_ptr(st[k]) for k in STATE_KEYS])


def init_state(prob) -> dict:
    """Initial iterate (zeros; x = Pi(0)) as a dict of float64 arrays."""
    H = _Holder(prob)
    m, q, n = H.m, H.q, H.n
    st = {"x": np.empty((m, q, n)), "z": np.empty((m, q, n)), "lam": np.empty((m, q, n)),
          "s": np.empty((q, n)), "mu": np.empty((q, n)), "h": np.empty((m, q)), "p": np.empty((m, q)),
          "nu": np.empty((m, q)), "x1": np.empty(m)}
    lib().orc_init_state(C.byref(H.c), C.byref(_state_struct(st)))
    return st


def solve(prob, par, state: dict | None = None, threads: int = 1, count_differs: bool = False):
    """Runs the iteration from ``state`` (default: the zero start) until the
    stop test or ``par.max_iter``.  Returns (state, report dict); the input
    state dict is not modified."""
    H = _Holder(prob)
    st = init_state(prob) if state is None else {k: _f64(state[k]).copy() for k in STATE_KEYS}
    rep = _Report()
    rc = lib().orc_solve(C.byref(H.c), C.byref(_params(par, threads, count_differs, H.n)),
                         C.byref(_state_struct(st)), C.byref(rep))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    out = {"iters": rep.iters, "converged": bool(rep.converged), "r": rep.r, "sigma": rep.sigma,
           "r_terms": list(rep.r_terms), "s_terms": list(rep.s_terms),
           "branch_count": list(rep.branch_count), "literal_differs": rep.literal_differs,
           "rho": list(rep.rho)}
    return st, out


def objective(prob, x) -> float:
    H = _Holder(prob)
    xx = _f64(x)
    return lib().orc_objective(C.byref(H.c), _ptr(xx))


def kkt(prob, par, state: dict):
    """KKT residual of eq. (2) at an iterate: (max, terms[8])."""
    H = _Holder(prob)
    st = {k: _f64(state[k]) for k in STATE_KEYS}
    t = np.zeros(8)
    v = lib().orc_kkt(C.byref(H.c), C.byref(_params(par, n=H.n)), C.byref(_state_struct(st)), _ptr(t))
    return v, t


def shard_phase_a(prob, par, state: dict, k0: int, xprev, sprev, threads: int = 1, n_total: int | None = None):
    """Phase A of the column-sharded iteration on a worker's slice ``prob``
    (its columns [k0, k0 + prob.n)): step (a), steps (e), (f), and the
    worker's record [2 m q + 2] (see orc_shard_phase_a).  ``state`` holds
    the worker's columns and every pair scalar; it is updated in place.
    Returns (g(x) [m, q, n_s], record)."""
    H = _Holder(prob)
    m, q, n = H.m, H.q, H.n
    gx = np.empty((m, q, n))
    colsum = np.empty((q, n))
    rec = np.empty(2 * m * q + 2)
    xp, sp = _f64(xprev), _f64(sprev)
    lib().orc_shard_phase_a(C.byref(H.c), C.byref(_params(par, threads, n=n_total or n)),
                            C.byref(_state_struct(state)), int(k0), _ptr(xp), _ptr(sp), _ptr(gx), _ptr(colsum),
                            _ptr(rec))
    return gx, rec


def shard_phase_b(prob, par, state: dict, n_total: int, tot, gx, zprev, hprev):
    """Phase B of the column-sharded iteration with the combined record
    ``tot``: steps (b), (g) on the worker's columns and (c), (d), (h), (i)
    on the pair scalars (see orc_shard_phase_b).  Returns the residual terms
    [|z - g(x)| max, |z - z~| max (the worker's), |h - 1'z|, copies,
    |h - h~| (every worker's)]."""
    H = _Holder(prob)
    res = np.empty(5)
    t, g, zp, hp = _f64(tot), _f64(gx), _f64(zprev), _f64(hprev)
    lib().orc_shard_phase_b(C.byref(H.c), C.byref(_params(par, n=n_total)), C.byref(_state_struct(state)),
                            int(n_total), _ptr(t), _ptr(g), _ptr(zp), _ptr(hp), _ptr(res))
    return res

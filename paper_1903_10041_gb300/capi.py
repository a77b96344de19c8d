"""Thin ctypes binding of the C ABI in ``include/admm.h`` (``libadmm.so``).

Argument marshalling only: every step of the solver runs in the CUDA
kernels of the library.  Arrays may be numpy arrays (host memory) or torch
CUDA tensors (device memory); both must be float64 and C-contiguous.
Importing this module raises ImportError when the library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# ADMM_LIB=debug loads the bounds-checked build (libadmm_debug.so) instead
LIB_PATH = os.path.join(HERE, "libadmm_debug.so" if os.environ.get("ADMM_LIB") == "debug" else "libadmm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1903_10041_gb300.build.build() "
                      "(or __graft_entry__.build()); there is no fallback path")

_lib = C.CDLL(LIB_PATH)
_dp = C.POINTER(C.c_double)

(ADMM_OK, ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA, ADMM_ETIMEOUT, ADMM_ENOTCONVERGED, ADMM_EUNSUPPORTED,
 ADMM_EPENDING, ADMM_ECANCELLED, ADMM_EBOUNDS) = range(10)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTCONVERGED",
                6: "EUNSUPPORTED", 7: "EPENDING", 8: "ECANCELLED", 9: "EBOUNDS"}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_fp64cubic": 2}
XMIN = {"exact": 0, "paper": 1}
SWEEP = {"gauss_seidel": 0, "jacobi": 1}
MAX_M = 8
MAX_PAIRS = 1024


class admm_problem(C.Structure):
    # the array pointers as c_void_p (the same ABI as const double *): they take the integer
    # address directly, which keeps marshalling thousands of problems cheap
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("q", C.c_int32),
                ("f2", C.c_void_p), ("f1", C.c_void_p), ("f0", C.c_void_p), ("g2", C.c_void_p),
                ("g1", C.c_void_p), ("g0", C.c_void_p), ("x_lo", C.c_void_p), ("x_hi", C.c_void_p),
                ("y", C.c_void_p), ("c", C.c_void_p), ("on_device", C.c_int32), ("coef_shared", C.c_int32)]


class admm_params(C.Structure):
    _fields_ = [("rho", C.c_double * 4), ("r_tol", C.c_double), ("s_tol", C.c_double), ("tau", C.c_double),
                ("max_iter", C.c_int32), ("check_every", C.c_int32), ("precision", C.c_int32),
                ("xmin_mode", C.c_int32), ("sweep", C.c_int32), ("adapt_rho", C.c_int32),
                ("rho2_over_n", C.c_int32), ("adapt_start", C.c_int32), ("reserved", C.c_int32 * 2)]


class admm_state(C.Structure):
    _fields_ = [("x", _dp), ("s", _dp), ("mu", _dp), ("lam", _dp), ("zeta", _dp), ("h", _dp), ("p", _dp),
                ("nu", _dp), ("x1", _dp), ("rho", C.c_double * 4), ("cold", C.c_int32),
                ("on_device", C.c_int32)]


class admm_result(C.Structure):
    _fields_ = [("x", _dp), ("x1", _dp), ("on_device", C.c_int32), ("iters", C.c_int32),
                ("converged", C.c_int32), ("status", C.c_int32), ("objective", C.c_double),
                ("r", C.c_double), ("sigma", C.c_double)]


_H = C.c_void_p
_lib.admm_default_params.argtypes = [C.POINTER(admm_params)]
_lib.admm_default_params.restype = None
_lib.admm_create.argtypes = [C.POINTER(admm_problem), C.POINTER(admm_params), C.POINTER(_H)]
_lib.admm_create.restype = C.c_int
_lib.admm_set_params.argtypes = [_H, C.POINTER(admm_params)]
_lib.admm_set_params.restype = C.c_int
_lib.admm_solve.argtypes = [_H, C.POINTER(admm_state), C.POINTER(admm_result), C.c_void_p]
_lib.admm_solve.restype = C.c_int
_lib.admm_wait.argtypes = [_H, C.POINTER(admm_result)]
_lib.admm_wait.restype = C.c_int
_lib.admm_reset.argtypes = [_H]
_lib.admm_reset.restype = C.c_int
_lib.admm_get_state.argtypes = [_H, C.POINTER(admm_state), C.c_void_p]
_lib.admm_get_state.restype = C.c_int
_lib.admm_destroy.argtypes = [_H]
_lib.admm_destroy.restype = C.c_int
_lib.admm_last_error.argtypes = []
_lib.admm_last_error.restype = C.c_char_p
_lib.admm_status_string.argtypes = [C.c_int]
_lib.admm_status_string.restype = C.c_char_p
_lib.admm_get_info.argtypes = [_H, _dp, C.c_int]
_lib.admm_get_info.restype = C.c_int
_lib.admm_selftest_barrier_timeout.argtypes = [C.c_longlong, C.c_int, C.POINTER(C.c_int)]
_lib.admm_selftest_barrier_timeout.restype = C.c_int
_lib.admm_selftest_bounds.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
_lib.admm_selftest_bounds.restype = C.c_int


class AdmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def admm_last_error() -> str:
    return _lib.admm_last_error().decode()


def _check(st: int, allow=(ADMM_OK,)) -> int:
    if st not in allow:
        raise AdmmError(st, admm_last_error())
    return st


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, keep: list):
    """Pointer to a float64 C-contiguous array; numpy (host) or torch (device)."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch tensors must be float64 and contiguous")
        keep.append(a)
        return C.cast(C.c_void_p(a.data_ptr()), _dp), bool(a.is_cuda)
    arr = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(arr)
    return arr.ctypes.data_as(_dp), False


def admm_default_params() -> admm_params:
    p = admm_params()
    _lib.admm_default_params(C.byref(p))
    return p


def make_params(par=None, **kw) -> admm_params:
    """admm_params from a duck-typed settings object (rho, r_tol, s_tol,
    max_iter, check_every, precision, xmin_mode, sweep, adapt_rho, tau, adapt_start)."""
    p = admm_default_params()
    src = {}
    if par is not None:
        for k in ("rho", "r_tol", "s_tol", "max_iter", "check_every", "precision", "xmin_mode", "sweep",
                  "adapt_rho", "tau", "rho2_over_n", "adapt_start"):
            if hasattr(par, k):
                src[k] = getattr(par, k)
    src.update(kw)
    if "rho" in src:
        for t in range(4):
            p.rho[t] = float(src["rho"][t])
    for k in ("r_tol", "s_tol", "tau"):
        if k in src:
            setattr(p, k, float(src[k]))
    for k in ("max_iter", "check_every", "adapt_start"):
        if k in src:
            setattr(p, k, int(src[k]))
    if "precision" in src:
        p.precision = PRECISION[src["precision"]] if isinstance(src["precision"], str) else int(src["precision"])
    if "xmin_mode" in src:
        p.xmin_mode = XMIN[src["xmin_mode"]] if isinstance(src["xmin_mode"], str) else int(src["xmin_mode"])
    if "sweep" in src:
        p.sweep = SWEEP[src["sweep"]] if isinstance(src["sweep"], str) else int(src["sweep"])
    if "adapt_rho" in src:
        p.adapt_rho = int(bool(src["adapt_rho"]))
    if "rho2_over_n" in src:
        p.rho2_over_n = int(bool(src["rho2_over_n"]))
    return p


def _addr(a, keep: list):
    """Address of a float64 C-contiguous array (numpy on the host, torch on either side)."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("torch tensors must be float64 and contiguous")
        keep.append(a)
        return a.data_ptr(), bool(a.is_cuda)
    arr = np.ascontiguousarray(a, dtype=np.float64)
    keep.append(arr)
    return arr.ctypes.data, False


def make_problem(prob, keep: list) -> admm_problem:
    """admm_problem pointing at the arrays of a duck-typed problem object."""
    names = ("f2", "f1", "f0", "g2", "g1", "g0", "lo", "hi", "y", "c")
    ptrs, devs = [], set()
    for nm in names:
        p, d = _addr(getattr(prob, nm), keep)
        ptrs.append(p)
        devs.add(d)
    if len(devs) != 1:
        raise TypeError("problem arrays must be all host or all device")
    return admm_problem(int(prob.n), int(prob.m), int(prob.q), *ptrs, int(devs.pop()),
                        int(bool(getattr(prob, "coef_shared", False))))


# ---------------------------------------------------------------------------
# the C ABI, same names
# ---------------------------------------------------------------------------
def admm_create(prob, par=None, **kw) -> C.c_void_p:
    keep: list = []
    cp = make_problem(prob, keep)
    pp = par if isinstance(par, admm_params) else make_params(par, **kw)
    h = _H()
    _check(_lib.admm_create(C.byref(cp), C.byref(pp), C.byref(h)))
    return h


def admm_set_params(h, par=None, **kw) -> None:
    pp = par if isinstance(par, admm_params) else make_params(par, **kw)
    _check(_lib.admm_set_params(h, C.byref(pp)))


def admm_reset(h) -> None:
    _check(_lib.admm_reset(h))


def _state_struct(st: dict, keep: list) -> admm_state:
    names = ("x", "s", "mu", "lam", "zeta", "h", "p", "nu", "x1")
    ptrs, devs = [], set()
    for nm in names:
        p, d = _ptr(st[nm], keep)
        ptrs.append(p)
        devs.add(d)
    if len(devs) != 1:
        raise TypeError("state arrays must be all host or all device")
    rho = (C.c_double * 4)(*[float(v) for v in st["rho"]])
    return admm_state(*ptrs, rho, int(bool(st.get("cold", False))), int(devs.pop()))


_ERRORS = (ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA, ADMM_ETIMEOUT, ADMM_EUNSUPPORTED)


class Pending:
    """A queued solve: keeps its result record and buffers alive until waited on."""

    def __init__(self, h, res, keep):
        self.h, self.res, self.keep = h, res, keep


def admm_solve_async(h, warm: dict | None = None, x_out=None, x1_out=None, stream=None) -> Pending:
    """Queues a solve (admm_solve) and returns without waiting for it.
    ``x_out``/``x1_out``: optional numpy or torch buffers that receive x
    [m, q, n] and x_1 [m].  ``stream``: a torch.cuda.Stream, an integer
    cudaStream_t, or None (legacy default stream)."""
    keep: list = []
    ws = C.byref(_state_struct(warm, keep)) if warm is not None else None
    res = admm_result()
    if x_out is not None or x1_out is not None:
        px, dx = _ptr(x_out, keep)
        p1, d1 = _ptr(x1_out, keep)
        res.x = px
        res.x1 = p1
        res.on_device = int(bool(dx or d1))
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    st = _lib.admm_solve(h, ws, C.byref(res), sp)
    if st != ADMM_OK:
        raise AdmmError(st, admm_last_error())
    return Pending(h, res, keep)


def admm_wait(pending: Pending, raise_on=_ERRORS) -> dict:
    """Waits for a queued solve and returns its outcome."""
    res = pending.res
    st = _lib.admm_wait(pending.h, C.byref(res))
    if st in raise_on:
        raise AdmmError(st, admm_last_error())
    return {"status": st, "iters": res.iters, "converged": bool(res.converged), "objective": res.objective,
            "r": res.r, "sigma": res.sigma}


def admm_solve(h, warm: dict | None = None, x_out=None, x1_out=None, stream=None, raise_on=_ERRORS) -> dict:
    """Runs a solve to its end: admm_solve, then admm_wait."""
    return admm_wait(admm_solve_async(h, warm, x_out, x1_out, stream), raise_on)


def admm_get_state(h, n: int, m: int, q: int) -> dict:
    """The handle's current state as numpy arrays (keys as in admm_state)."""
    st = {"x": np.empty((m, q, n)), "s": np.empty((q, n)), "mu": np.empty((q, n)),
          "lam": np.empty((m, q)), "zeta": np.empty((m, q)), "h": np.empty((m, q)), "p": np.empty((m, q)),
          "nu": np.empty((m, q)), "x1": np.empty(m), "rho": [0.0] * 4, "cold": False}
    keep: list = []
    cs = _state_struct(st, keep)
    _check(_lib.admm_get_state(h, C.byref(cs), None))
    st["rho"] = [cs.rho[t] for t in range(4)]
    st["cold"] = bool(cs.cold)
    return st


INFO_KEYS = ("iters", "converged", "r", "sigma", "r_demand", "r_z", "r_h", "r_copy", "s_z", "s_h", "s_sx",
             "objective", "status", "fp64_escalations")


def admm_get_info(h) -> dict:
    """Per-solve record of the last solve on the handle (see admm.h)."""
    buf = (C.c_double * 16)()
    _check(_lib.admm_get_info(h, buf, 16))
    return {k: buf[t] for t, k in enumerate(INFO_KEYS)}


def admm_destroy(h) -> None:
    if h:
        _lib.admm_destroy(h)


def admm_selftest_barrier_timeout(spin_ns: int = 20_000_000, grid: int = 4) -> int:
    out = C.c_int(-1)
    _check(_lib.admm_selftest_barrier_timeout(int(spin_ns), int(grid), C.byref(out)))
    return out.value


def admm_selftest_bounds():
    """(status, index) of the checked build's bounds self-test (admm.h)."""
    st, ix = C.c_int(-1), C.c_longlong(-1)
    _check(_lib.admm_selftest_bounds(C.byref(st), C.byref(ix)))
    return st.value, ix.value


def quartic_min(A, B, Cc, D, lo, hi, mode: str = "exact", precision: str = "fp64", stream=None, out=None):
    """Algorithm 1 + clamp on many quartics (admm_quartic_min[_f32]).  The
    six inputs are 1-D arrays of one length: numpy (host; copied inside the
    call) or CUDA torch tensors (device).  precision "fp64" (float64 arrays)
    or "fp32" (float32 arrays).  Returns x (numpy or torch, like the inputs)."""
    f32 = precision == "fp32"
    arrs = [A, B, Cc, D, lo, hi]
    if _is_torch(A):
        import torch
        dt = torch.float32 if f32 else torch.float64
        for a in arrs:
            if a.dtype != dt or not a.is_contiguous() or not a.is_cuda:
                raise TypeError("tensors must be contiguous CUDA tensors of the precision's dtype")
        x = out if out is not None else torch.empty_like(A)
        ptrs = [C.c_void_p(a.data_ptr()) for a in arrs + [x]]
        dev = 1
    else:
        dt = np.float32 if f32 else np.float64
        arrs = [np.ascontiguousarray(a, dtype=dt) for a in arrs]
        x = out if out is not None else np.empty_like(arrs[0])
        ptrs = [a.ctypes.data_as(C.c_void_p) for a in arrs + [x]]
        dev = 0
    n = int(arrs[0].shape[0])
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    fn = _lib.admm_quartic_min_f32 if f32 else _lib.admm_quartic_min
    st = fn(*ptrs[:6], C.c_int64(n), ptrs[6], int(XMIN[mode]), int(dev), sp)
    if st != ADMM_OK:
        raise AdmmError(st, admm_last_error())
    return x


class Solver:
    """Owns one handle: ``Solver(problem, params).solve()``."""

    def __init__(self, prob, par=None, **kw):
        self._pending = None
        self.n, self.m, self.q = int(prob.n), int(prob.m), int(prob.q)
        self.h = admm_create(prob, par, **kw)

    def solve(self, warm=None, **kw) -> dict:
        return admm_solve(self.h, warm, **kw)

    def solve_async(self, warm=None, **kw) -> Pending:
        """Queues a solve on ``stream`` and returns at once; ``wait`` ends it."""
        self._pending = admm_solve_async(self.h, warm, **kw)
        return self._pending

    def wait(self, **kw) -> dict:
        p, self._pending = self._pending, None
        return admm_wait(p, **kw)

    def set_params(self, par=None, **kw):
        admm_set_params(self.h, par, **kw)

    def reset(self):
        admm_reset(self.h)

    def state(self) -> dict:
        return admm_get_state(self.h, self.n, self.m, self.q)

    def info(self) -> dict:
        return admm_get_info(self.h)

    def close(self):
        if self.h:
            admm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_lib.admm_solve_noalloc.argtypes = [C.POINTER(admm_problem), C.POINTER(admm_params), C.POINTER(admm_state),
                                    C.POINTER(admm_result), C.c_void_p]
_lib.admm_solve_noalloc.restype = C.c_int


def admm_solve_noalloc(prob_dev, par, state_dev: dict, x_out=None, x1_out=None, stream=None,
                       raise_on=(ADMM_EINVAL, ADMM_ENOMEM, ADMM_ECUDA, ADMM_ETIMEOUT, ADMM_EUNSUPPORTED)) -> dict:
    """The allocation-free solve: ``prob_dev`` and ``state_dev`` hold torch
    CUDA tensors (float64, contiguous); ``state_dev`` is updated in place
    (its "rho" and "cold" entries too).  See admm_solve_noalloc in admm.h."""
    keep: list = []
    cp = make_problem(prob_dev, keep)
    pp = par if isinstance(par, admm_params) else make_params(par)
    cs = _state_struct(state_dev, keep)
    res = admm_result()
    if x_out is not None or x1_out is not None:
        px, dx = _ptr(x_out, keep)
        p1, d1 = _ptr(x1_out, keep)
        res.x, res.x1, res.on_device = px, p1, int(bool(dx or d1))
    sp = None
    if stream is not None:
        sp = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    st = _lib.admm_solve_noalloc(C.byref(cp), C.byref(pp), C.byref(cs), C.byref(res), sp)
    if st in raise_on:
        raise AdmmError(st, admm_last_error())
    state_dev["rho"] = [cs.rho[t] for t in range(4)]
    state_dev["cold"] = bool(cs.cold)
    return {"status": st, "iters": res.iters, "converged": bool(res.converged), "objective": res.objective,
            "r": res.r, "sigma": res.sigma}


# ---------------------------------------------------------------------------
# batched solves
# ---------------------------------------------------------------------------
class admm_batch_config(C.Structure):
    _fields_ = [("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32), ("small_max_elements", C.c_int64),
                ("cluster_size", C.c_int32), ("reserved", C.c_int32), ("cluster_min_elements", C.c_int64)]


_B = C.c_void_p
_lib.admm_batch_create.argtypes = [C.POINTER(admm_problem), C.c_int32, C.POINTER(admm_params), C.POINTER(_B)]
_lib.admm_batch_set_config.argtypes = [_B, C.POINTER(admm_batch_config)]
_lib.admm_batch_get_config.argtypes = [_B, C.POINTER(admm_batch_config)]
_lib.admm_batch_autotune.argtypes = [_B, C.c_int32, C.POINTER(admm_batch_config)]
_lib.admm_batch_solve.argtypes = [_B, C.c_void_p]
_lib.admm_batch_wait.argtypes = [_B, C.c_void_p, C.POINTER(admm_result)]
_lib.admm_batch_get_info.argtypes = [_B, C.c_int32, _dp, C.c_int32]
_lib.admm_batch_get_state.argtypes = [_B, C.c_int32, C.POINTER(admm_state)]
_lib.admm_batch_set_state.argtypes = [_B, C.c_int32, C.POINTER(admm_state)]
_lib.admm_batch_reset.argtypes = [_B]
_lib.admm_batch_destroy.argtypes = [_B]
for _f in ("admm_batch_create", "admm_batch_set_config", "admm_batch_get_config", "admm_batch_autotune",
           "admm_batch_solve", "admm_batch_wait", "admm_batch_get_info", "admm_batch_get_state",
           "admm_batch_set_state", "admm_batch_reset", "admm_batch_destroy"):
    getattr(_lib, _f).restype = C.c_int


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def _cfg_dict(c: admm_batch_config) -> dict:
    return {"warps_per_cta": c.warps_per_cta, "ctas_per_sm": c.ctas_per_sm,
            "small_max_elements": c.small_max_elements, "cluster_size": c.cluster_size,
            "cluster_min_elements": c.cluster_min_elements}


class Batch:
    """Many instances solved together (admm_batch_* in admm.h); mixed precision."""

    def __init__(self, problems, par=None, **kw):
        self._keep: list = []
        self.shapes = [(int(p.n), int(p.m), int(p.q)) for p in problems]
        arr = (admm_problem * len(problems))(*[make_problem(p, self._keep) for p in problems])
        pp = par if isinstance(par, admm_params) else make_params(par, **kw)
        if pp.precision != PRECISION["mixed"]:
            pp.precision = PRECISION["mixed"]
        self.h = _B()
        _check(_lib.admm_batch_create(arr, len(problems), C.byref(pp), C.byref(self.h)))
        self._keep = []  # the batch holds its own copy of the data
        self.count = len(problems)

    def set_config(self, warps_per_cta=8, ctas_per_sm=0, small_max_elements=0, cluster_size=1,
                   cluster_min_elements=131072):
        c = admm_batch_config(int(warps_per_cta), int(ctas_per_sm), int(small_max_elements), int(cluster_size), 0,
                              int(cluster_min_elements))
        _check(_lib.admm_batch_set_config(self.h, C.byref(c)))

    def config(self) -> dict:
        c = admm_batch_config()
        _check(_lib.admm_batch_get_config(self.h, C.byref(c)))
        return _cfg_dict(c)

    def autotune(self, trial_iters: int = 30) -> dict:
        c = admm_batch_config()
        _check(_lib.admm_batch_autotune(self.h, int(trial_iters), C.byref(c)))
        return _cfg_dict(c)

    def solve(self, stream=None):
        _check(_lib.admm_batch_solve(self.h, _stream_ptr(stream)))

    def wait(self, stream=None, want_x: bool = False) -> list:
        res = (admm_result * self.count)()
        xs = []
        if want_x:
            for t, (n, m, q) in enumerate(self.shapes):
                x = np.empty((m, q, n))
                x1 = np.empty(m)
                xs.append((x, x1))
                res[t].x = x.ctypes.data_as(_dp)
                res[t].x1 = x1.ctypes.data_as(_dp)
                res[t].on_device = 0
        st = _lib.admm_batch_wait(self.h, _stream_ptr(stream), res)
        if st not in (ADMM_OK, ADMM_ENOTCONVERGED):
            raise AdmmError(st, admm_last_error())
        out = []
        for t in range(self.count):
            d = {"status": res[t].status, "iters": res[t].iters, "converged": bool(res[t].converged),
                 "objective": res[t].objective, "r": res[t].r, "sigma": res[t].sigma}
            if want_x:
                d["x"], d["x1"] = xs[t]
            out.append(d)
        return out

    def info(self, idx: int) -> dict:
        buf = (C.c_double * 16)()
        _check(_lib.admm_batch_get_info(self.h, int(idx), buf, 16))
        return {k: buf[t] for t, k in enumerate(INFO_KEYS)}

    def state(self, idx: int) -> dict:
        n, m, q = self.shapes[idx]
        st = {"x": np.empty((m, q, n)), "s": np.empty((q, n)), "mu": np.empty((q, n)),
              "lam": np.empty((m, q)), "zeta": np.empty((m, q)), "h": np.empty((m, q)), "p": np.empty((m, q)),
              "nu": np.empty((m, q)), "x1": np.empty(m), "rho": [0.0] * 4, "cold": False}
        keep: list = []
        cs = _state_struct(st, keep)
        _check(_lib.admm_batch_get_state(self.h, int(idx), C.byref(cs)))
        st["rho"] = [cs.rho[t] for t in range(4)]
        st["cold"] = bool(cs.cold)
        return st

    def set_state(self, idx: int, st: dict):
        keep: list = []
        cs = _state_struct(st, keep)
        _check(_lib.admm_batch_set_state(self.h, int(idx), C.byref(cs)))

    def reset(self):
        _check(_lib.admm_batch_reset(self.h))

    def close(self):
        if self.h:
            _lib.admm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
class admm_server_config(C.Structure):
    _fields_ = [("store_elements", C.c_int64), ("max_active", C.c_int32), ("tick_iters", C.c_int32),
                ("max_m", C.c_int32), ("max_q", C.c_int32), ("batch", admm_batch_config)]


_S = C.c_void_p
_lib.admm_server_default_config.argtypes = [C.POINTER(admm_server_config)]
_lib.admm_server_default_config.restype = None
_lib.admm_server_create.argtypes = [C.POINTER(admm_params), C.POINTER(admm_server_config), C.POINTER(_S)]
_lib.admm_server_submit.argtypes = [_S, C.POINTER(admm_problem), C.c_int64, C.POINTER(C.c_int64)]
_lib.admm_server_poll.argtypes = [_S, C.c_int64, C.c_int32, C.POINTER(admm_result), _dp]
_lib.admm_server_stats.argtypes = [_S, _dp, C.c_int32]
_lib.admm_server_destroy.argtypes = [_S]
for _f in ("admm_server_create", "admm_server_submit", "admm_server_poll", "admm_server_stats",
           "admm_server_destroy"):
    getattr(_lib, _f).restype = C.c_int


class admm_step(C.Structure):
    _fields_ = [("m", C.c_int32), ("q", C.c_int32), ("f2", _dp), ("f1", _dp), ("f0", _dp), ("g2", _dp),
                ("g1", _dp), ("g0", _dp), ("x_lo", _dp), ("x_hi", _dp), ("y", _dp)]


_lib.admm_server_submit_step.argtypes = [_S, C.c_int64, C.POINTER(admm_step), C.POINTER(C.c_int64)]
_lib.admm_server_drain.argtypes = [_S, C.c_int32, C.POINTER(C.c_int64), _dp, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.admm_server_drain.restype = C.c_int
_lib.admm_server_submit_step.restype = C.c_int


class Server:
    """Continuous-batching request loop (admm_server_* in admm.h).

    Requests are whole problems (``submit``) or receding-horizon steps of a
    session whose instance stays resident on the device (``submit_step``).
    A worker thread admits queued requests in arrival order into a device
    store of ``store_elements`` elements (an instance takes m*q*ld, ld = n
    rounded up to 4; at most ``max_active`` instances at once) and runs
    ticks: one launch of the batched kernel over every active instance, in
    which the costliest instance runs ``tick_iters`` iterations and the
    others a time-balanced share.  Finished instances leave at the tick
    boundary, so a request's result does not depend on which others shared
    its ticks.  ``cancel`` ends a request with ADMM_ECANCELLED; ``poll`` and
    ``drain`` return results; ``stats`` reports counters and GPU time.
    Requests solve in the mixed-precision path.
    """

    def __init__(self, par=None, store_elements=1 << 27, max_active=4096, tick_iters=10, max_m=4, max_q=20,
                 warps_per_cta=8, ctas_per_sm=0, small_max_elements=0, cluster_size=1,
                 cluster_min_elements=131072, **kw):
        pp = par if isinstance(par, admm_params) else make_params(par, **kw)
        pp.precision = PRECISION["mixed"]
        cfg = admm_server_config()
        _lib.admm_server_default_config(C.byref(cfg))
        cfg.store_elements, cfg.max_active, cfg.tick_iters = int(store_elements), int(max_active), int(tick_iters)
        cfg.max_m, cfg.max_q = int(max_m), int(max_q)
        cfg.batch = admm_batch_config(int(warps_per_cta), int(ctas_per_sm), int(small_max_elements),
                                      int(cluster_size), 0, int(cluster_min_elements))
        self.h = _S()
        _check(_lib.admm_server_create(C.byref(pp), C.byref(cfg), C.byref(self.h)))
        self._shapes = {}
        self._session_n = {}

    def submit_step(self, session: int, step: dict) -> int:
        """Receding-horizon step request (admm_server_submit_step): ``step``
        holds f2, f1, f0, g2, g1, g0 [m, q], lo, hi [m] and y [q]."""
        keep: list = []
        m, q = step["f2"].shape
        ptrs = [_ptr(step[k], keep)[0] for k in ("f2", "f1", "f0", "g2", "g1", "g0", "lo", "hi", "y")]
        cs = admm_step(int(m), int(q), *ptrs)
        t = C.c_int64()
        _check(_lib.admm_server_submit_step(self.h, int(session), C.byref(cs), C.byref(t)))
        n = self._session_n.get(int(session))
        self._shapes[t.value] = (n if n is not None else 0, int(m), int(q))
        return t.value

    def submit(self, prob, session: int = -1) -> int:
        keep: list = []
        cp = make_problem(prob, keep)
        t = C.c_int64()
        _check(_lib.admm_server_submit(self.h, C.byref(cp), int(session), C.byref(t)))
        self._shapes[t.value] = (int(prob.n), int(prob.m), int(prob.q))
        if session >= 0:
            self._session_n[int(session)] = int(prob.n)
        return t.value

    def cancel(self, ticket: int) -> None:
        """admm_server_cancel: the request finishes with ADMM_ECANCELLED."""
        _check(_lib.admm_server_cancel(self.h, C.c_int64(int(ticket))))

    def poll(self, ticket: int, wait_ms: int = 0, want_x: bool = False):
        """None while pending; else a result dict (with x, x1 if want_x)."""
        if ticket not in self._shapes:
            raise AdmmError(ADMM_EINVAL, f"unknown or already returned ticket {ticket}")
        n, m, q = self._shapes[ticket]
        res = admm_result()
        x = x1 = None
        if want_x:
            x, x1 = np.empty((m, q, n)), np.empty(m)
            res.x, res.x1 = x.ctypes.data_as(_dp), x1.ctypes.data_as(_dp)
        times = (C.c_double * 3)()
        st = _lib.admm_server_poll(self.h, int(ticket), int(wait_ms), C.byref(res), times)
        if st == ADMM_EPENDING:
            return None
        del self._shapes[ticket]
        d = {"status": res.status if st == ADMM_OK else st, "iters": res.iters, "converged": bool(res.converged),
             "objective": res.objective, "r": res.r, "sigma": res.sigma, "admit_s": times[0],
             "latency_s": times[1], "warm": bool(times[2])}
        if want_x:
            d["x"], d["x1"] = x, x1
        return d

    def drain(self, max_count: int = 65536):
        """Finished requests as (tickets, latency_s, iters, status) numpy arrays."""
        t = np.empty(max_count, dtype=np.int64)
        lat = np.empty(max_count)
        it = np.empty(max_count, dtype=np.int32)
        st = np.empty(max_count, dtype=np.int32)
        cnt = C.c_int32()
        _check(_lib.admm_server_drain(self.h, int(max_count), t.ctypes.data_as(C.POINTER(C.c_int64)),
                                      lat.ctypes.data_as(_dp), it.ctypes.data_as(C.POINTER(C.c_int32)),
                                      st.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(cnt)))
        k = cnt.value
        for tk in t[:k]:
            self._shapes.pop(int(tk), None)
        return t[:k], lat[:k], it[:k], st[:k]

    def stats(self) -> dict:
        buf = (C.c_double * 10)()
        _check(_lib.admm_server_stats(self.h, buf, 10))
        keys = ("ticks", "admitted", "finished", "active", "queued", "store_free_frac", "sessions", "gpu_busy_s",
                "gpu_shift_s", "instance_ticks")
        return {k: buf[t] for t, k in enumerate(keys)}

    def close(self):
        if self.h:
            _lib.admm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

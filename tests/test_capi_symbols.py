"""The C-ABI library builds, loads and exports every function that
include/*.h declares.  CPU only: no compute call is made."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(hdr).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(admm_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1903_10041_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("admm_create", "admm_solve", "admm_destroy", "admm_get_state", "admm_set_params",
                 "admm_default_params", "admm_last_error"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_bounds_checked_build_exports_the_same_symbols():
    """libadmm_debug.so (-DADMM_DEBUG_BOUNDS) is the same boundary with the
    element accesses checked."""
    from paper_1903_10041_gb300 import build
    dbg = ctypes.CDLL(build.build(debug_bounds=True))
    missing = [n for n in sorted(_declared()) if not hasattr(dbg, n)]
    assert not missing, missing


def test_host_only_calls_work_without_a_gpu():
    from paper_1903_10041_gb300 import capi
    p = capi.admm_default_params()
    assert p.max_iter == 5000 and p.check_every == 10 and abs(p.tau - 1.1) < 1e-15
    assert list(p.rho) == [1.0, 1.0, 1.0, 1.0]
    # NULL handle and NULL arguments are rejected without touching the device
    assert capi._lib.admm_solve(None, None, None, None) == capi.ADMM_EINVAL
    assert capi._lib.admm_destroy(None) == capi.ADMM_OK
    assert capi._lib.admm_create(None, None, None) == capi.ADMM_EINVAL


def test_struct_layouts_match_the_header(lib):
    """ctypes mirrors of the C structs have the sizes the header implies."""
    from paper_1903_10041_gb300 import capi
    assert ctypes.sizeof(capi.admm_params) == 8 * 7 + 4 * 6 + 4 * 4
    assert ctypes.sizeof(capi.admm_problem) == 16 + 8 * 10 + 8
    assert ctypes.sizeof(capi.admm_state) == 8 * 9 + 8 * 4 + 8


def test_binding_refuses_to_load_without_the_library(tmp_path):
    """No CPU fallback: the binding raises ImportError when libadmm.so is
    absent beside it, instead of running anything else."""
    import importlib.util
    import shutil
    src = os.path.join(ROOT, "paper_1903_10041_gb300", "capi.py")
    shutil.copy(src, tmp_path / "capi.py")
    spec = importlib.util.spec_from_file_location("capi_without_lib", tmp_path / "capi.py")
    mod = importlib.util.module_from_spec(spec)
    with pytest.raises(ImportError, match="no fallback"):
        spec.loader.exec_module(mod)


def test_status_codes_match_the_header():
    from paper_1903_10041_gb300 import capi
    txt = open(os.path.join(ROOT, "include", "admm.h")).read()
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ADMM_[A-Z]+)\s*=\s*(\d+)", txt)}
    for name in ("ADMM_OK", "ADMM_EINVAL", "ADMM_ENOMEM", "ADMM_ECUDA", "ADMM_ETIMEOUT", "ADMM_ENOTCONVERGED",
                 "ADMM_EUNSUPPORTED", "ADMM_EPENDING", "ADMM_ECANCELLED", "ADMM_EBOUNDS"):
        assert getattr(capi, name) == codes[name], name
        assert capi.STATUS_NAMES[codes[name]] == name[len("ADMM_"):]


def test_batch_and_server_creation_validate_on_the_host():
    """Bad arguments are refused before any device call (no GPU needed)."""
    from paper_1903_10041_gb300 import capi
    p = capi.admm_default_params()
    p.precision = capi.PRECISION["mixed"]
    cfg = capi.admm_server_config()
    capi._lib.admm_server_default_config(ctypes.byref(cfg))
    h = capi._S()
    assert capi._lib.admm_server_create(None, ctypes.byref(cfg), ctypes.byref(h)) == capi.ADMM_EINVAL
    for field, bad in (("reserved", 1), ("small_max_elements", -1), ("cluster_size", 3), ("warps_per_cta", 6)):
        c2 = capi.admm_server_config()
        ctypes.pointer(c2)[0] = cfg
        setattr(c2.batch, field, bad)
        assert capi._lib.admm_server_create(ctypes.byref(p), ctypes.byref(c2), ctypes.byref(h)) == capi.ADMM_EINVAL
        assert not h.value
    for field, bad in (("max_active", 0), ("tick_iters", 0), ("max_m", capi.MAX_M + 1)):
        c2 = capi.admm_server_config()
        ctypes.pointer(c2)[0] = cfg
        setattr(c2, field, bad)
        assert capi._lib.admm_server_create(ctypes.byref(p), ctypes.byref(c2), ctypes.byref(h)) == capi.ADMM_EINVAL
    p64 = capi.admm_default_params()  # FP64: the server runs the mixed path only
    assert capi._lib.admm_server_create(ctypes.byref(p64), ctypes.byref(cfg), ctypes.byref(h)) == \
        capi.ADMM_EUNSUPPORTED
    b = capi._B()
    assert capi._lib.admm_batch_create(None, 1, ctypes.byref(p), ctypes.byref(b)) == capi.ADMM_EINVAL
    assert capi._lib.admm_batch_destroy(None) == capi.ADMM_OK
    assert capi._lib.admm_server_destroy(None) == capi.ADMM_OK


def test_plain_c_client_builds_and_runs(lib, tmp_path):
    """The boundary is usable from C99 alone: tests/c_abi_host.c compiles
    against include/admm.h, links libadmm.so and makes the host-only calls."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    so = lib._name
    exe = tmp_path / "c_abi_host"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_host.c"), so, "-lm",
                    "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert "c client ok" in out.stdout


def test_create_refuses_bad_sizes_and_settings_on_the_host():
    """Empty and oversized instances and bad settings are refused by
    admm_create before it touches a device (no GPU needed), with the
    status the header documents."""
    from paper_1903_10041_gb300 import capi
    from paper_1903_10041_gb300 import workloads as W

    def create(prob, par=None, edit=None):
        keep: list = []
        cp = capi.make_problem(prob, keep)
        if edit:
            edit(cp)
        pp = par or capi.admm_default_params()
        h = capi._H()
        st = capi._lib.admm_create(ctypes.byref(cp), ctypes.byref(pp), ctypes.byref(h))
        assert not h.value
        return st

    P = W.random_problem(4, 2, 1, seed=3)
    assert create(P, edit=lambda c: setattr(c, "n", 0)) == capi.ADMM_EINVAL       # empty horizon
    assert create(P, edit=lambda c: setattr(c, "q", 0)) == capi.ADMM_EINVAL       # no scenario
    assert create(W.random_problem(3, capi.MAX_M + 1, 1, seed=3)) == capi.ADMM_EUNSUPPORTED
    assert create(W.random_problem(2, 1, capi.MAX_PAIRS + 1, seed=3)) == capi.ADMM_EUNSUPPORTED
    assert create(P, edit=lambda c: setattr(c, "y", None)) == capi.ADMM_EINVAL
    assert create(P, edit=lambda c: setattr(c, "coef_shared", 2)) == capi.ADMM_EINVAL

    def par(**kw):
        p = capi.admm_default_params()
        for k, v in kw.items():
            if k == "rho1":
                p.rho[1] = v
            elif k == "reserved":
                p.reserved[0] = v
            else:
                setattr(p, k, v)
        return p

    for kw in ({"rho1": 0.0}, {"rho1": float("inf")}, {"r_tol": float("nan")}, {"max_iter": 0},
               {"check_every": 0}, {"xmin_mode": 5}, {"sweep": 3}, {"adapt_rho": 1, "tau": 1.0}, {"adapt_start": -1},
               {"reserved": 1}):
        assert create(P, par(**kw)) == capi.ADMM_EINVAL, kw
    assert create(P, par(precision=9)) == capi.ADMM_EUNSUPPORTED
    assert "precision" in capi.admm_last_error()


def test_server_poll_of_an_unknown_ticket_is_an_error():
    """A ticket the binding never issued (or already returned) is refused
    before any call into the library."""
    from paper_1903_10041_gb300 import capi
    s = object.__new__(capi.Server)
    s.h, s._shapes, s._session_n = None, {}, {}
    with pytest.raises(capi.AdmmError) as e:
        s.poll(12345)
    assert e.value.status == capi.ADMM_EINVAL


def test_batch_and_server_refuse_bad_settings_before_any_device_call():
    """Batches and servers check their settings first (the rules of
    admm_create: adapt_start >= 0, tolerances >= 0, reserved fields 0) and a
    server refuses a store beyond the kernel's 32-bit array offsets; none of
    this needs a device."""
    from paper_1903_10041_gb300 import capi
    from paper_1903_10041_gb300 import workloads as W
    P = W.random_problem(4, 2, 1, seed=3)
    keep = []
    cp = capi.make_problem(P, keep)

    def mixed(**kw):
        pp = capi.make_params(W.Params(precision="mixed"))
        for k, v in kw.items():
            if k == "reserved":
                pp.reserved[0] = v
            else:
                setattr(pp, k, v)
        return pp

    for kw in ({"adapt_start": -1}, {"reserved": 1}, {"r_tol": -1.0}):
        h = capi._B()
        st = capi._lib.admm_batch_create(ctypes.byref(cp), 1, ctypes.byref(mixed(**kw)), ctypes.byref(h))
        assert st == capi.ADMM_EINVAL and not h.value, kw
    cfg = capi.admm_server_config()
    capi._lib.admm_server_default_config(ctypes.byref(cfg))
    s = capi._S()
    assert capi._lib.admm_server_create(ctypes.byref(mixed(adapt_start=-1)), ctypes.byref(cfg),
                                        ctypes.byref(s)) == capi.ADMM_EINVAL and not s.value
    cfg.store_elements = 1 << 32
    assert capi._lib.admm_server_create(ctypes.byref(mixed()), ctypes.byref(cfg),
                                        ctypes.byref(s)) == capi.ADMM_EUNSUPPORTED and not s.value
    assert "32-bit" in capi.admm_last_error()

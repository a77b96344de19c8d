"""The bounds-checked build (libadmm_debug.so, -DADMM_DEBUG_BOUNDS): every
element access of the mixed element update is checked against its
instance's arrays and an access outside them is recorded (ADMM_EBOUNDS)
instead of faulting.  Its self-test records an index past a buffer without
touching memory outside it; on the batched recipe (CTA and cluster teams,
shared and per-scenario maps) and a single-instance solve it records
nothing and gives the release build's bits."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def _run(tmp_path, lib):
    path = os.path.join(str(tmp_path), f"{lib}.npz")
    env = dict(os.environ, ADMM_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_debug_bounds_child.py"), path],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return dict(np.load(path))


def test_checked_build_records_nothing_and_matches_the_release_build(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    build.build(debug_bounds=True)
    from paper_1903_10041_gb300 import capi
    dbg, rel = _run(tmp_path, "debug"), _run(tmp_path, "release")
    assert dbg["selftest"][0] == capi.ADMM_EBOUNDS and dbg["selftest"][1] == 20
    assert rel["selftest"][0] == -capi.ADMM_EUNSUPPORTED       # the release build has no checks
    keys = [k for k in rel if k != "selftest"]
    assert len(keys) == 12
    for k in keys:
        if k.endswith("iters"):
            assert dbg[k][1] in (capi.ADMM_OK, capi.ADMM_ENOTCONVERGED), (k, dbg[k])
        assert np.array_equal(dbg[k], rel[k]), k

"""The product path and the oracle share no code: nothing in the package
(Python binding, CUDA sources) or the public header refers to the oracle,
nothing in the oracle refers to the solver library or its header (the only
module both sides use is the seeded input generator).  Checked on the
source text and on the loaded library.  CPU only."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _read(paths):
    return {p: open(p, encoding="utf-8").read() for p in paths}


def test_product_sources_never_refer_to_the_oracle():
    pkg = os.path.join(ROOT, "paper_1903_10041_gb300")
    files = (glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*")) +
             glob.glob(os.path.join(ROOT, "include", "*.h")))
    for path, txt in _read(files).items():
        if path.endswith("workloads.py"):
            # the shared input generator may say that both sides use it, nothing more
            assert not re.search(r"import\s+oracle|from\s+oracle|liboracle|orc_", txt), path
            continue
        assert not re.search(r"\boracle\b|liboracle|orc_", txt), path


def test_oracle_sources_never_refer_to_the_solver_library():
    hdr = open(os.path.join(ROOT, "include", "admm.h"), encoding="utf-8").read()
    api = set(re.findall(r"\b(admm_[a-z_]+)\s*\(", re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)))
    assert "admm_solve" in api and "admm_create" in api
    files = glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "oracle", "*.c"))
    for path, txt in _read(files).items():
        assert not re.search(r"paper_1903_10041_gb300|libadmm|admm\.h", txt), path
        used = {name for name in api if re.search(r"\b" + name + r"\b", txt)}
        assert not used, (path, used)


def test_library_exports_no_oracle_symbol():
    from paper_1903_10041_gb300 import build
    lib = ctypes.CDLL(build.build())
    for name in ("orc_solve", "orc_quartic_min", "orc_kkt", "orc_objective"):
        assert not hasattr(lib, name), name

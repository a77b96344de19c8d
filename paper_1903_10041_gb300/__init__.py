"""GB300-native parallel ADMM for robust quadratic resource allocation.

The solver is a C-ABI CUDA library (``libadmm.so``, declared in
``include/admm.h``); :mod:`paper_1903_10041_gb300.capi` is its thin ctypes
binding.  :mod:`paper_1903_10041_gb300.workloads` generates seeded inputs.
Submodules are imported lazily so that the input generators can be used on
machines where the library has not been built.
"""
import importlib

__all__ = ["capi", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

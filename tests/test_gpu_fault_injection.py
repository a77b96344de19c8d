"""Host-side fault injection (no GPU fault): ADMM_FAULT_ALLOC = k makes the
k-th device allocation of admm_create fail.  Every such create returns
ADMM_ENOMEM, frees what it had allocated, and the next create works."""
import os

import pytest

from paper_1903_10041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_allocation_failures_in_create_leave_nothing_behind(capi, precision):
    import torch
    P = W.random_problem(100_000, 2, 4, seed=31)  # 6.4 MB per FP64 array: a leak would show
    par = W.Params(rho=(1.0, 1.0 / P.n, 1.0, 1.0), precision=precision, max_iter=20)
    with capi.Solver(P, par) as s:  # warm up the context and allocator
        s.solve(raise_on=(1, 2, 3, 4, 6))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    try:
        for k in range(1, 19):
            os.environ["ADMM_FAULT_ALLOC"] = str(k)
            with pytest.raises(capi.AdmmError) as ei:
                capi.Solver(P, par)
            assert ei.value.status == capi.ADMM_ENOMEM, k
    finally:
        del os.environ["ADMM_FAULT_ALLOC"]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < 32 << 20, (free0 - free1)
    with capi.Solver(P, par) as s:
        assert s.solve(raise_on=(1, 2, 3, 4, 6))["iters"] == 20

"""Quartic benchmark entry points (Sec. III-C): Algorithm 1 + clamp on many
independent quartics, FP64 and FP32, host and device arrays, against the
oracle's minimiser (Algorithm 1 in FP64, same inputs)."""
import numpy as np
import pytest

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


def quartics(n, seed):
    """Single and double wells (about a third double), some A = 0, random
    intervals; exactly representable in FP32."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.01, 2.0, n)
    A[rng.random(n) < 0.05] = 0.0
    B = rng.uniform(-2.0, 2.0, n)
    Cc = rng.uniform(-3.0, 3.0, n)
    Cc[A == 0.0] = np.abs(Cc[A == 0.0]) + 0.1
    D = rng.uniform(-2.0, 2.0, n)
    c0, w = rng.uniform(-2.0, 2.0, n), rng.uniform(0.0, 3.0, n)
    lo, hi = c0 - w, c0 + w
    return [v.astype(np.float32).astype(np.float64) for v in (A, B, Cc, D, lo, hi)]


def F(A, B, Cc, D, x):
    return ((A * x + B) * x + Cc) * x * x + D * x


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_fp64_matches_the_oracle(capi, oracle_lib, mode):
    A, B, Cc, D, lo, hi = quartics(200_001, seed=11)
    x_o, br = oracle_lib.quartic_min(A, B, Cc, D, lo, hi, mode=mode)
    x_g = capi.quartic_min(A, B, Cc, D, lo, hi, mode=mode)
    assert (br == 2).mean() > 0.1 and (br == 3).mean() > 0.01  # trig and quadratic branches present
    f_o, f_g = F(A, B, Cc, D, x_o), F(A, B, Cc, D, x_g)
    assert np.all(f_g <= f_o + 1e-10 * (1.0 + np.abs(f_o)))
    close = np.abs(x_g - x_o) <= 1e-9 * np.maximum(1.0, np.abs(x_o))
    assert close.mean() > 0.9999, close.mean()  # the rest are ties between two equal minima


def test_fp32_matches_the_oracle_to_fp32_accuracy(capi, oracle_lib):
    A, B, Cc, D, lo, hi = quartics(100_003, seed=12)
    x_o, _ = oracle_lib.quartic_min(A, B, Cc, D, lo, hi)
    x_g = capi.quartic_min(*[v.astype(np.float32) for v in (A, B, Cc, D, lo, hi)], precision="fp32")
    x_g = x_g.astype(np.float64)
    f_o, f_g = F(A, B, Cc, D, x_o), F(A, B, Cc, D, x_g)
    assert np.all(f_g <= f_o + 1e-5 * (1.0 + np.abs(f_o)))
    assert (np.abs(x_g - x_o) <= 1e-4 * np.maximum(1.0, np.abs(x_o))).mean() > 0.999


def test_device_arrays_and_invalid_elements(capi, oracle_lib):
    import torch
    A, B, Cc, D, lo, hi = quartics(4097, seed=13)
    dev = [torch.from_numpy(v).cuda() for v in (A, B, Cc, D, lo, hi)]
    x_d = capi.quartic_min(*dev).cpu().numpy()
    assert np.array_equal(x_d, capi.quartic_min(A, B, Cc, D, lo, hi))
    A_bad = A.copy()
    A_bad[[5, 77]] = -1.0
    with pytest.raises(capi.AdmmError) as ei:
        capi.quartic_min(A_bad, B, Cc, D, lo, hi)
    assert ei.value.status == capi.ADMM_EINVAL


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_fp64_acos_clamp_case(capi, oracle_lib, mode):
    """The cubic of the oracle's acos-clamp pin (subnormal R^2, the computed
    argument of acos 1 + 5e-10): the GPU's FP64 minimiser clamps it too and
    returns the oracle's finite minimiser."""
    from tests.test_oracle_quartic import ACOS_CLAMP_CUBIC
    b, c, d = ACOS_CLAMP_CUBIC
    args = [np.array([v]) for v in (0.25, b, c / 2.0, d, -1.0, 1.0)]
    x = capi.quartic_min(*args, mode=mode, precision="fp64")
    xo, br = oracle_lib.quartic_min(*[a[0] for a in args], mode=mode)
    assert br == 2 and np.isfinite(x[0]) and abs(x[0] - float(xo)) <= 1e-9 * abs(float(xo)), (x[0], xo)

"""The GPU's FP64 quartic minimiser (Algorithm 1 + the clamp of step (a),
the entry point of the Sec. III-C benchmark) against the exact minimisers of
tests/golden/quartic_cases.txt, which come from factorised derivatives in
rational arithmetic, not from the oracle.  No quartic value may exceed the
exact minimum; the position must match to 1e-9 except at the exact tie
(two equal minima, either is right) and at triple roots, whose flat minimum
fixes the position only to about the cube root of the rounding."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_10041_gb300 import build
    build.build()
    from paper_1903_10041_gb300 import capi
    return capi


def test_fp64_minimiser_meets_the_exact_cases(capi):
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "quartic_cases.txt")) if not ln.startswith("#")]
    br = np.array([int(r[0]) for r in rows])
    v = np.array([[float(t) for t in r[1:]] for r in rows])
    A, B, C, D, lo, hi, want = (np.ascontiguousarray(v[:, t]) for t in range(7))
    x = capi.quartic_min(A, B, C, D, lo, hi)

    def F(z):
        return ((A * z + B) * z + C) * z * z + D * z

    assert np.all(F(x) <= F(want) + 1e-12 * (1.0 + np.abs(F(want))))
    tie = (A == 1.0) & (B == 0.0) & (C == -2.0) & (D == 0.0)
    strict = (br != 1) & ~tie
    assert strict.sum() >= 80
    err = np.abs(x - want) / np.maximum(1.0, np.abs(want))
    assert err[strict].max() <= 1e-9, (np.argmax(np.where(strict, err, 0)), err[strict].max())
    assert np.abs(x[br == 1] - want[br == 1]).max() <= 1e-4

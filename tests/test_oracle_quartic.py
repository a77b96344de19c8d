"""Pins of the oracle's quartic minimiser (Algorithm 1, Sec. III-B) against
closed forms, constructed roots and brute force.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

from tests._independent import quartic_argmin_grid, quartic_value


def _coeffs_from_roots(A, r1, r2, r3):
    """f'(x) = 4A (x - r1)(x - r2)(x - r3) = 4A x^3 + 3B x^2 + 2C x + D."""
    e1, e2, e3 = r1 + r2 + r3, r1 * r2 + r1 * r3 + r2 * r3, r1 * r2 * r3
    return A, -4 * A * e1 / 3, 2 * A * e2, -4 * A * e3


def test_cubic_roots_trig_branch_recovers_constructed_roots(oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(200):
        r = np.sort(rng.uniform(-5, 5, 3))
        if np.min(np.diff(r)) < 0.05:
            continue
        b, c, d = -(r.sum()), r[0] * r[1] + r[0] * r[2] + r[1] * r[2], -np.prod(r)
        roots, br = oracle_lib.cubic_roots(b, c, d)
        assert br == 2
        assert np.allclose(np.sort(roots), r, atol=1e-11, rtol=0)


def test_cubic_roots_cardano_single_real_root(oracle_lib):
    rng = np.random.default_rng(1)
    for _ in range(200):
        # (x - r)(x^2 + px + s) with p^2 < 4s: one real root r
        r, p = rng.uniform(-5, 5, 2)
        s = p * p / 4 + rng.uniform(0.1, 10)
        b, c, d = p - r, s - r * p, -r * s
        roots, br = oracle_lib.cubic_roots(b, c, d)
        assert br == 0 and len(roots) == 1
        assert abs(roots[0] - r) <= 1e-11 * max(1, abs(r))


def test_triple_root_takes_vieta_branch(oracle_lib):
    # (x - r)^4 = x^4 - 4r x^3 + 6r^2 x^2 - 4r^3 x + r^4; dyadic r keeps Q = R = 0 exact
    for r in (0.5, -1.25, 2.0, 0.0):
        x, br = oracle_lib.quartic_min(1.0, -4 * r, 6 * r * r, -4 * r ** 3)
        assert br == 1 and x == r


def test_quadratic_branch_when_A_is_zero(oracle_lib):
    x, br = oracle_lib.quartic_min(0.0, 0.0, 2.0, -3.0)          # 2x^2 - 3x -> 0.75
    assert br == 3 and x == 0.75
    x, br = oracle_lib.quartic_min(0.0, 0.0, 2.0, -3.0, -1.0, 0.5)
    assert x == 0.5


def test_symmetric_double_well_tie_keeps_smaller_root(oracle_lib):
    # x^4 - 2x^2: minima at -1 and 1 with equal values; Algorithm 1 keeps x_1
    for mode in ("exact", "paper"):
        x, br = oracle_lib.quartic_min(1.0, 0.0, -2.0, 0.0, mode=mode)
        assert br == 2 and abs(x + 1.0) < 1e-12


def test_constructed_double_well_picks_lower_minimum_exactly(oracle_lib):
    """Rational roots: the lower well is decided in exact arithmetic."""
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(300):
        num = rng.integers(-40, 41, 3)
        if len(set(num)) < 3:
            continue
        r1, r2, r3 = sorted(Fraction(int(v), 8) for v in num)
        A = Fraction(int(rng.integers(1, 9)), 4)
        Af, Bf, Cf, Df = _coeffs_from_roots(A, r1, r2, r3)
        F = lambda x: Af * x ** 4 + Bf * x ** 3 + Cf * x ** 2 + Df * x
        if F(r1) == F(r3):
            continue
        want = r1 if F(r1) < F(r3) else r3
        x, br = oracle_lib.quartic_min(float(Af), float(Bf), float(Cf), float(Df))
        assert br == 2
        assert abs(x - float(want)) <= 1e-10 * max(1.0, abs(float(want)))
        checked += 1
    assert checked > 200


@pytest.mark.parametrize("seed", [3, 4])
def test_random_quartics_on_intervals_match_grid_search(oracle_lib, seed):
    """Exact mode: the clamped result is the constrained minimiser (grid + Newton)."""
    rng = np.random.default_rng(seed)
    cnt = 300
    A = rng.uniform(0.01, 2.0, cnt)
    B, Cc, D = rng.uniform(-5, 5, (3, cnt))
    lo = rng.uniform(-4, 1, cnt)
    hi = lo + rng.uniform(0.1, 5, cnt)
    x, br = oracle_lib.quartic_min(A, B, Cc, D, lo, hi, mode="exact")
    assert set(np.unique(br)) <= {0, 2}
    for t in range(cnt):
        xb, fb, gap = quartic_argmin_grid(A[t], B[t], Cc[t], D[t], lo[t], hi[t])
        fo = quartic_value(A[t], B[t], Cc[t], D[t], x[t])
        scale = max(1.0, abs(fb))
        assert lo[t] <= x[t] <= hi[t]
        assert fo <= fb + 1e-12 * scale, (t, x[t], xb)
        if gap > 1e-9 * scale:
            assert abs(x[t] - xb) <= 1e-7 * max(1.0, abs(xb)), (t, x[t], xb)


def test_paper_mode_clamps_the_global_minimiser(oracle_lib):
    """Roots -1.5, 0, 2 with the deeper well at 2; on [-2, 1] the literal
    Pi(argmin) gives 1, while the constrained minimiser is -1.5."""
    A, B, Cc, D = _coeffs_from_roots(1.0, -1.5, 0.0, 2.0)
    F = lambda x: quartic_value(A, B, Cc, D, x)
    assert F(2.0) < F(-1.5) and F(-1.5) < F(1.0)
    xp, _ = oracle_lib.quartic_min(A, B, Cc, D, -2.0, 1.0, mode="paper")
    xe, _ = oracle_lib.quartic_min(A, B, Cc, D, -2.0, 1.0, mode="exact")
    assert xp == 1.0
    assert abs(xe + 1.5) < 1e-12
    # both agree when the interval holds the global minimiser
    xp, _ = oracle_lib.quartic_min(A, B, Cc, D, -2.0, 3.0, mode="paper")
    xe, _ = oracle_lib.quartic_min(A, B, Cc, D, -2.0, 3.0, mode="exact")
    assert abs(xp - 2.0) < 1e-12 and xp == xe


def _golden_quartics():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "quartic_cases.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    br = np.array([int(r[0]) for r in rows])
    v = np.array([[float(t) for t in r[1:]] for r in rows])
    return br, v


def test_golden_quartics_with_exact_minimisers(oracle_lib):
    """tests/golden/quartic_cases.txt: minimisers fixed by factorised
    derivatives in exact arithmetic, every branch of Algorithm 1 with and
    without clamping, double roots of the cubic (Delta = 0, decided either
    way by rounding) and the exact tie of the symmetric double well."""
    br, v = _golden_quartics()
    assert set(br.tolist()) == {-1, 0, 1, 2, 3} and len(br) >= 90
    x, branch = oracle_lib.quartic_min(*[v[:, t] for t in range(6)])
    want = v[:, 6]
    fixed = br >= 0  # a double root (-1) may round to either the Cardano or the trig branch
    assert np.array_equal(branch[fixed], br[fixed])
    assert np.isin(branch[~fixed], (0, 2)).all()
    assert np.abs(x - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


# A cubic x^3 + b x^2 + c x + d whose computed Delta is 0 (trig branch) while
# R / sqrt(-Q^3) rounds to 1 + 5e-10: R^2 and Q^3 lie in the subnormal range.
# In binary64 with correctly rounded square root and division the argument
# cannot pass +-1 when the computed Delta <= 0 unless R^2 or Q^3 is
# subnormal (fl(sqrt(fl(x*x))) = |x| otherwise), so the case has to sit there.
ACOS_CLAMP_CUBIC = (0.0, -3.3729653494511964e-105, -7.539906031043884e-158)


def test_acos_argument_clamp_is_needed_in_the_subnormal_range(oracle_lib):
    """Reading R6: the argument of acos in the trig branch of Algorithm 1 is
    clamped to [-1, 1].  On this cubic the unclamped argument exceeds 1 in
    binary64, so without the clamp the roots are NaN; with it they are the
    double root -sqrt(-Q) and the simple root 2 sqrt(-Q) (theta = 0)."""
    b, c, d = ACOS_CLAMP_CUBIC
    # the case really exercises the clamp (Python floats are binary64)
    Q = c / 3.0 - b * b / 9.0
    R = b * c / 6.0 - b * b * b / 27.0 - d / 2.0
    assert Q * Q * Q + R * R <= 0.0 and abs(R / math.sqrt(-Q * Q * Q)) > 1.0
    roots, branch = oracle_lib.cubic_roots(b, c, d)
    assert branch == 2 and np.all(np.isfinite(roots)), roots
    s = math.sqrt(-Q)
    np.testing.assert_allclose(np.sort(roots), [-s, -s, 2.0 * s], rtol=1e-7)
    # each root makes the cubic vanish to the rounding of its terms
    for r in roots:
        assert abs(r ** 3 + c * r + d) <= 1e-6 * abs(d)
    # the quartic with this derivative (A = 1/4: b = B, c = 2 C, d = D) has a finite minimiser
    x, br = oracle_lib.quartic_min(0.25, b, c / 2.0, d, -1.0, 1.0)
    assert br == 2 and math.isfinite(float(x)) and abs(float(x) - 2.0 * s) <= 1e-7 * s

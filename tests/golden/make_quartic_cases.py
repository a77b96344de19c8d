"""Writes quartic_cases.txt: quartics with known constrained minimisers.

Each case is built from the factorisation of the derivative, so the answer
follows from the mathematics, not from any solver:

    f(x) = A x^4 + B x^3 + C x^2 + D x,   f'(x) = 4A x^3 + 3B x^2 + 2C x + D.

- three real roots r1 < r2 < r3:  f'(x) = 4A (x - r1)(x - r2)(x - r3);
- a double root r and a simple t: f'(x) = 4A (x - r)^2 (x - t);
- one real root r:                f'(x) = 4A (x - r)(x^2 + p x + s), p^2 < 4s;
- triple root r:                  f(x) = A (x - r)^4 minus its constant;
- quadratic (A = B = 0):          f(x) = C x^2 + D x, C > 0.

With A = 3 alpha and dyadic alpha and roots, every coefficient is a dyadic
rational with a short numerator, so it is exact in binary64.  The minimiser
over [lo, hi] is found in exact rational arithmetic among lo, hi and the real
roots of f' inside the interval; equal values keep the smaller point (the
tie rule of Algorithm 1, Sec. III-B, kept after clamping).  The branch
column names the case of Algorithm 1 the cubic f'/4A falls in: 0 one real
root (Delta > 0, Cardano), 1 triple root (Q = R = 0), 2 three real roots
(trigonometric form), 3 quadratic (A = 0), -1 a double root (Delta = 0 in
exact arithmetic, so rounding sends it to either the Cardano or the
trigonometric branch).

Run from the repository root:  python tests/golden/make_quartic_cases.py
"""
import os
import random
from fractions import Fraction as Fr

HERE = os.path.dirname(os.path.abspath(__file__))


def f(x, A, B, C, D):
    return ((A * x + B) * x + C) * x * x + D * x


def argmin(A, B, C, D, lo, hi, roots):
    cands = sorted({lo, hi} | {r for r in roots if lo < r < hi})
    vals = [f(x, A, B, C, D) for x in cands]
    best = min(vals)
    # smallest point attaining the minimum; reject near ties a binary64
    # comparison could flip
    second = min([v for v in vals if v != best], default=None)
    return cands[vals.index(best)], (second - best if second is not None else None)


def dy(rng, lo, hi, den):
    return Fr(rng.randint(lo * den, hi * den), den)


def main():
    rng = random.Random(1903)
    rows = []

    def add(kind, A, B, C, D, lo, hi, roots):
        x, gap = argmin(A, B, C, D, lo, hi, roots)
        scale = max(1, abs(f(lo, A, B, C, D)), abs(f(hi, A, B, C, D)))
        if gap is not None and gap / scale < Fr(1, 10**6):
            return False
        rows.append((kind, A, B, C, D, lo, hi, x))
        return True

    def interval(roots):
        while True:
            lo, hi = sorted((dy(rng, -4, 4, 4), dy(rng, -4, 4, 4)))
            if lo < hi:
                return lo, hi

    n3 = 0
    while n3 < 40:  # three distinct real roots
        r1, r2, r3 = sorted(dy(rng, -3, 3, 8) for _ in range(3))
        if not (r1 + Fr(1, 8) <= r2 and r2 + Fr(1, 8) <= r3):
            continue
        al = Fr(rng.randint(1, 8), 4)
        A = 3 * al
        e1, e2, e3 = r1 + r2 + r3, r1 * r2 + r1 * r3 + r2 * r3, r1 * r2 * r3
        lo, hi = interval((r1, r2, r3))
        n3 += add(2, A, -4 * al * e1, 6 * al * e2, -12 * al * e3, lo, hi, (r1, r2, r3))
    n1 = 0
    while n1 < 20:  # one real root
        r, p = dy(rng, -3, 3, 8), dy(rng, -2, 2, 4)
        s = p * p / 4 + Fr(rng.randint(1, 16), 8)
        al = Fr(rng.randint(1, 8), 4)
        A = 3 * al
        lo, hi = interval((r,))
        n1 += add(0, A, 4 * al * (p - r), 6 * al * (s - r * p), -12 * al * r * s, lo, hi, (r,))
    n2 = 0
    while n2 < 24:  # a double root of f' (a saddle of f) and a simple one (the minimum)
        r, t = dy(rng, -3, 3, 8), dy(rng, -3, 3, 8)
        if abs(r - t) < Fr(1, 4):
            continue
        al = Fr(rng.randint(1, 8), 4)
        A = 3 * al
        # f'(x) = 4A (x - r)^2 (x - t): roots r (double), t
        e1, e2, e3 = 2 * r + t, r * r + 2 * r * t, r * r * t
        lo, hi = interval((r, t))
        n2 += add(-1, A, -4 * al * e1, 6 * al * e2, -12 * al * e3, lo, hi, (r, t))
    for _ in range(8):  # triple root: A (x - r)^4, A a power of two
        r, A = dy(rng, -3, 3, 4), Fr(2) ** rng.randint(-2, 2)
        lo, hi = interval((r,))
        add(1, A, -4 * A * r, 6 * A * r * r, -4 * A * r ** 3, lo, hi, (r,))
    for _ in range(8):  # quadratic
        Cq, xs = Fr(rng.randint(1, 16), 4), dy(rng, -3, 3, 8)
        lo, hi = interval((xs,))
        add(3, Fr(0), Fr(0), Cq, -2 * Cq * xs, lo, hi, (xs,))
    # the symmetric double well x^4 - 2x^2: an exact tie kept on the smaller root
    rows.append((2, Fr(1), Fr(0), Fr(-2), Fr(0), Fr(-3), Fr(3), Fr(-1)))

    with open(os.path.join(HERE, "quartic_cases.txt"), "w") as fh:
        fh.write("# Quartics A x^4 + B x^3 + C x^2 + D x on [lo, hi] with their exact minimiser x*\n"
                 "# (Algorithm 1, Sec. III-B, and the clamp of step (a), App. A; ties keep the smaller\n"
                 "# point).  Written by make_quartic_cases.py from factorised derivatives in exact\n"
                 "# rational arithmetic; every value is exact in binary64 (repr round-trips).\n"
                 "# branch A B C D lo hi x*\n")
        for kind, *vals in rows:
            assert all(float(v) == v for v in vals)
            fh.write(" ".join([str(kind)] + [repr(float(v)) for v in vals]) + "\n")
    print(f"{len(rows)} cases")


if __name__ == "__main__":
    main()

"""The FP64 quotient of the force of infection: a float reciprocal seed, two Newton-Raphson
steps and Markstein's remainder correction (each step a fused multiply-add).  Evaluated
here with exact rational arithmetic for every FMA and a float32 reciprocal as the seed
(the hardware approximation is within one float ulp; both seeds are far inside the
method's basin), it must stay within one ulp of the correctly rounded quotient for
divisors across the range the kernels use, and equal it in nearly all cases.  The GPU
kernels are checked against the FP64 oracle by the parity tests; this pins the method."""
from fractions import Fraction

import numpy as np


def _fma(a, b, c):
    """a * b + c with one rounding (exact rational product and sum, then the nearest double)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _quotient(num, d):
    r = float(np.float32(1.0) / np.float32(d))  # float reciprocal seed
    r = _fma(r, _fma(-d, r, 1.0), r)
    r = _fma(r, _fma(-d, r, 1.0), r)
    q = num * r
    return _fma(r, _fma(-d, q, num), q)


def _ulps(a, b):
    ia = np.array([a], dtype=np.float64).view(np.int64)[0]
    ib = np.array([b], dtype=np.float64).view(np.int64)[0]
    return abs(int(ia) - int(ib))


def test_newton_markstein_quotient_is_within_one_ulp():
    g = np.random.Generator(np.random.PCG64(2603))
    n = 4000
    d = 10.0 ** g.uniform(-29, 29, n)              # inside the seed's range (1e-30, 1e30)
    d[: n // 4] = g.uniform(0.05, 2.0, n // 4)     # the densities the workloads produce
    num = d * g.uniform(0.0, 1.0, n) * 10.0 ** g.uniform(-8, 0, n)
    exact_ties = 0
    for a, b in zip(num, d):
        q = _quotient(float(a), float(b))
        want = float(Fraction(float(a)) / Fraction(float(b)))  # correctly rounded
        u = _ulps(q, want)
        assert u <= 1, (a, b, q, want)
        exact_ties += u == 0
    assert exact_ties >= n - 4, exact_ties


def test_special_values():
    assert _quotient(0.0, 1.0) == 0.0
    assert _quotient(3.0, 1.0) == 3.0
    assert _quotient(1.0, 3.0) == 1.0 / 3.0
    assert _quotient(0.25, 0.5) == 0.5

"""Pins of the oracle's incomplete Gamma function (App. C).

G(n,z) = Gamma(n) gamma*(n,z) = int_0^1 s^(n-1) e^(-zs) ds is checked against
the exact integer-n identity gamma(n,z) = (n-1)! [1 - e^-z sum_{k<n} z^k/k!]
evaluated in 1500-digit arithmetic (mpmath), which no cancellation reaches at
these sizes, and against special cases that reduce to elementary functions.
"""
import cmath
import math

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")


def G_exact(n, z):
    with mp.workdps(1500):
        z = mp.mpc(z)
        if z == 0:
            return complex(mp.mpf(1) / n)
        s, t = mp.mpf(0), mp.mpf(1)
        for k in range(n):
            if k:
                t = t * z / k
            s += t
        return complex(mp.factorial(n - 1) * (1 - mp.exp(-z) * s) / z ** n)


@pytest.mark.parametrize("n", [1, 2, 7, 41, 103, 140])
def test_G_matches_exact_identity(oracle, n):
    worst = 0.0
    branches = set()
    for r in [0.0, 0.4, 2.0, 9.0, 35.0, 80.0, 150.0, 260.0]:
        for ang in np.linspace(-np.pi, np.pi, 13):
            z = r * np.exp(1j * ang)
            g, br = oracle.G(n, z)
            branches.add(br)
            ref = G_exact(n, z)
            worst = max(worst, abs(g - ref) / abs(ref))
    assert worst < 5e-14, worst
    # every one of the four expansions is exercised for moderate n
    if n >= 7:
        assert branches == {"a", "b", "c", "d"}


def test_G_special_cases(oracle):
    # G(1,z) = (1 - e^-z)/z
    for z in [0.3 + 0.1j, -5 + 2j, 40j, 120 - 3j, -200 + 0.0j]:
        g, _ = oracle.G(1, z)
        assert abs(g - (1 - cmath.exp(-z)) / z) <= 1e-14 * abs(g)
    # G(n,0) = 1/n
    for n in [1, 5, 60]:
        assert abs(oracle.G(n, 0)[0] - 1.0 / n) < 1e-16
    # real z > 0: G(n,x) = Gamma(n) P(n,x) / x^n with scipy's regularised gamma
    sp = pytest.importorskip("scipy.special")
    for n in [3, 30, 90]:
        for x in [0.5, 10.0, 60.0, 200.0]:
            ref = math.exp(math.lgamma(n) - n * math.log(x)) * sp.gammainc(n, x)
            assert abs(oracle.G(n, x)[0] - ref) <= 1e-13 * ref
    # P(n,z) -> 1 for large Re z > 0
    assert abs(oracle.P(4, 80.0 + 5j) - 1.0) < 1e-14

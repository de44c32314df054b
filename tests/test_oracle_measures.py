"""Pins of the oracle's non-Markovian measures (App. D) and of the one-excitation
photon field phi(x,t) they use, against what the paper and the mathematics fix:

* phi(x,t) (not printed in the paper; read from the structure of Eq. 2 and the
  delay equation of the one-excitation sector) must conserve the
  one-excitation probability: |e0(t)|^2 + int |phi(x,t)|^2 dx = 1 when the
  incident packet is normalised.  A wrong sign or weight of either emission
  term breaks this at O(Gamma).
* At t = 0 the discrete definitions reduce to closed forms: psi(x > -a, 0) = 0,
  e1(0) = 1, e0(0) = 0, so mu(0) = lambda(0) = 1 + delta alpha Gamma / 2 (the
  trapezoid's first node carries |phi0(-a)|^2 = alpha Gamma with weight 1/2).
* With the coupling switched (almost) off the photon just moves and the atom
  just rotates: mu(t) -> e^{-i w0 t}, lambda(t) -> 1 (a conjugation on the wrong
  factor gives e^{+i w0 t}; a missing x <= -a part gives 1 - e^{-alpha Gamma t}).
* The measures converge as the grid is refined (first order: the packet has a
  sharp front).
"""
import math

import numpy as np
import pytest

import workloads as W


def stim(O, nx, nt, D, a=0.5, gamma=1.0, k0a=math.pi / 2, alpha=0.7, dk=0.3):
    w0 = k0a / a
    return O.Params(nx=nx, nt=nt, D=D, delta=2 * a / D, gamma=gamma, omega0=w0, k=w0 + dk, init_cond=2,
                    alpha=alpha)


def gl_integral(f, lo, hi, n=120):
    x, w = np.polynomial.legendre.leggauss(n)
    xm, xr = 0.5 * (hi + lo), 0.5 * (hi - lo)
    return sum(wi * f(xm + xr * xi) for xi, wi in zip(x, w)) * xr


@pytest.mark.parametrize("t", [0.7, 2.3, 4.1])
def test_one_excitation_probability_is_conserved(oracle, t):
    p = stim(oracle, 64, 64, 20, a=0.5, alpha=0.7, dk=0.3)
    a = p.a
    # phi(x,t) is smooth between the points where a gate switches (x = -a, a, t - a, t + a)
    # and where e0 at the retarded times t - x -+ a has a kink (its n-th term switches on
    # at 2na): x = t - a - 2na, t + a - 2na
    cuts = {-a, a, t - a, t + a}
    for n in range(1, int(t / (2 * a)) + 2):
        cuts |= {t - a - 2 * n * a, t + a - 2 * n * a}
    cuts = sorted(c for c in cuts if -a <= c <= t + a)
    inside = sum(gl_integral(lambda x: abs(oracle.phi1(p, x, t)) ** 2, lo, hi)
                 for lo, hi in zip(cuts[:-1], cuts[1:]))
    left = math.exp(-p.alpha * p.gamma * t)  # int_{-inf}^{-a} |phi0(x - t)|^2 dx
    total = abs(oracle.e0_one(p, t)) ** 2 + left + inside
    assert abs(total - 1.0) < 1e-10, total
    # the same sum with the sign of the mirror image's emission flipped is far from 1
    g = math.sqrt(0.5 * p.gamma)

    def flipped(x):
        v = oracle.phi1(p, x, t)
        if x > a and t - x + a > 0:
            v -= 2 * g * oracle.e0_one(p, t - x + a)
        return abs(v) ** 2
    bad = sum(gl_integral(flipped, lo, hi) for lo, hi in zip(cuts[:-1], cuts[1:]))
    if t > 2 * a:  # the mirror term has reached a region of width t - ... > 0
        assert abs(abs(oracle.e0_one(p, t)) ** 2 + left + bad - 1.0) > 1e-3


def test_measures_at_t0_closed_form(oracle):
    p = stim(oracle, 200, 50, 20)
    out = oracle.march(p, tstep=7)
    m = oracle.measures(p, out, tstep=7)
    want = 1.0 + 0.5 * p.delta * p.alpha * p.gamma
    assert abs(complex(m[0, 0], m[0, 1]) - want) < 1e-14
    assert abs(m[0, 2] - want) < 1e-14
    assert abs(m[0, 3] - want ** 3) < 1e-13


def test_measures_uncoupled_limit(oracle):
    # Gamma = 1e-6: mu(t) = e^{-i w0 t} and lambda(t) = 1 up to O(Gamma t)
    a, D = 0.5, 20
    p = stim(oracle, 600, 400, D, a=a, gamma=1e-6, alpha=1.0, dk=0.0)
    out = oracle.march(p, tstep=99)
    m = oracle.measures(p, out, tstep=99)
    for s, row in enumerate(m):
        t = s * 100 * p.delta
        assert abs(complex(row[0], row[1]) - np.exp(-1j * p.omega0 * t)) < 1e-4, (t, row)
        assert abs(row[2] - 1.0) < 1e-4


def test_measures_converge_on_refinement(oracle):
    # mu and lambda at t = 2.4 on three grids; the box covers the light cone x = t + a
    t, a = 2.4, 0.5
    vals = []
    for D in (20, 40, 80):
        delta = 2 * a / D
        n = int(round(t / delta))
        nx = int(round((t + 2 * a) / delta)) + D
        p = stim(oracle, nx, n + 1, D, a=a, alpha=1.0, dk=0.2)
        out = oracle.march(p, tstep=n)
        m = oracle.measures(p, out, tstep=n)
        vals.append(np.array([complex(m[-1, 0], m[-1, 1]), m[-1, 2]]))
    d1 = np.abs(vals[0] - vals[1])
    d2 = np.abs(vals[1] - vals[2])
    assert np.all(d2 < d1)
    assert np.all(d1 / d2 > 1.5) and np.all(d1 / d2 < 5.0), d1 / d2
    assert abs(vals[2][0]) < 1.0 + 1e-2 and 0.0 < vals[2][1] < 1.0 + 1e-2

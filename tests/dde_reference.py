"""Independent reference for the one-excitation amplitude e(t): direct
numerical integration of the delay equation that the closed forms of Sec. 2
solve,

    de/dt = -W e + (Gamma/2) e(t-2a) theta(t-2a) + s(t),   W = i w0 + Gamma/2,
    s(t)  = sqrt(Gamma/2) [phi(-a-t) - phi(a-t)],

by the method of steps: on each interval [2ja, 2(j+1)a] the delayed value is
the dense output of the previous interval, and the ODE is integrated with
scipy's DOP853 at rtol 1e-13.  All breakpoints of the drive and of the delay
fall on the interval ends.  Test-only; it shares nothing with the oracle but
the wavepacket phi, which it evaluates itself.
"""
from __future__ import annotations

import numpy as np
from scipy.integrate import solve_ivp


def phi_exp(x, k, alpha, gamma, a):
    ag = alpha * gamma
    return 1j * np.sqrt(ag) * np.exp(1j * k * x + 0.5 * ag * (x + a)) if x <= -a else 0.0


def phi_plane(x, k, a):
    return np.exp(1j * k * x) if x <= -a else 0.0


def phi_gauss(x, k, sigma, center, a):
    if x > -a:
        return 0.0
    return (2 * np.pi * sigma ** 2) ** -0.25 * np.exp(1j * k * x - (x - center) ** 2 / (4 * sigma ** 2))


def solve(a, gamma, omega0, T, phi=None, e0=0.0):
    W = 0.5 * gamma + 1j * omega0
    sols = []

    def delayed(t):
        s = t - 2 * a
        if s <= 0 or not sols:
            return 0.0
        j = min(int(s // (2 * a)), len(sols) - 1)
        return sols[j](s)[0]

    def drive(t):
        if phi is None:
            return 0.0
        return np.sqrt(gamma / 2) * (phi(-a - t) - phi(a - t))

    y = np.array([e0], dtype=complex)
    t0 = 0.0
    while t0 < T - 1e-14:
        t1 = min(t0 + 2 * a, T)
        f = lambda t, y: np.array([-W * y[0] + 0.5 * gamma * delayed(t) + drive(t)])
        r = solve_ivp(f, (t0, t1), y, method="DOP853", rtol=1e-13, atol=1e-15, dense_output=True)
        sols.append(r.sol)
        y = r.y[:, -1]
        t0 = t1

    def ev(t):
        j = min(int(t // (2 * a)), len(sols) - 1)
        return complex(sols[j](t)[0])

    return ev

"""Pins of the oracle's march (Eq. 1 discretised by Eq. 3a-c and Eq. 4).

* Validation test 1 of Sec. 4: marched inside x <= -a, the scheme reproduces
  the exact psi(x<-a,t) = C phi(x-t) e(t) at second order (this pins the
  square stencil, the delay term of App. A, the chi source and the boundary).
* Two-excitation probability: int |psi|^2 dx + int int |chi|^2 = 1, with chi
  rebuilt from the marched psi by Eq. 2 (the oracle's orc_chi).  This pins the
  mirror source terms (lines 2-3 of Eq. 1), which validation test 1 does not
  reach (flipping the sign of either one moves the total to ~4.6 or ~9), and
  orc_chi itself: a wrong weight or sign of either term of Eq. 2 breaks the sum.
* Causality: column m depends on nothing to the right of max(m, D/2), so a
  narrower box gives the same values on the common columns.
* Stability (App. A): long runs stay bounded.
* App. B unit conversions reproduce the printed caption values.
"""
import json
import math
import os

import numpy as np
import pytest

PI = math.pi
HERE = os.path.dirname(os.path.abspath(__file__))


def P(O, D, nrows, nx, ic=3, dk=0.0, alpha=1.0, **kw):
    dl = 2.0 / D
    return O.Params(nx=nx, nt=nrows, D=D, delta=dl, gamma=1.0, omega0=PI / 2, k=PI / 2 + dk, init_cond=ic,
                    alpha=alpha, **kw)


@pytest.mark.parametrize("ic,kw", [(1, {}), (1, dict(dk=0.3)), (2, {}), (3, {}), (3, dict(dk=0.4, alpha=0.7)),
                                   (4, dict(sigma=0.8, center=-1.0 - 6.4)),
                                   (5, dict(dk=0.3, alpha=0.7, k2=PI / 2 - 0.5, alpha2=1.4))])
def test_validation_left_second_order(oracle, ic, kw):
    errs = []
    for D in (20, 40, 80):
        dl = 2.0 / D
        nrows = int(round(6.0 / dl)) + 1
        L = int(round(3.0 / dl))
        p = P(oracle, D, nrows, D + 2, ic=ic, **kw)
        g = oracle.march_left(p, nrows, L)
        cols = np.arange(-D // 2 - L + 1, -D // 2 + 1)
        ex = np.array([oracle.psi_exact(p, nrows - 1, c) for c in cols])
        errs.append(np.linalg.norm(g[-1] - ex) / np.linalg.norm(ex))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.85, (errs, orders)


def total_probability(O, D, t_end=8.0, dk=0.0, alpha=1.0, Ltail=20.0):
    """int |psi|^2 + int int |chi|^2 at t_end, chi from Eq. 2 (two identical
    exponential photons; phi evaluated here, independently of the oracle)."""
    dl = 2.0 / D
    Dh = D // 2
    n = int(round(t_end / dl))
    nx = n + D + 4
    p = P(O, D, n + 1, nx, ic=3, dk=dk, alpha=alpha)
    res = O.march(p, n + 1, tstep=0, want_etab=True)
    grid, et, nrm = res["snaps"], res["etab"], res["norms"]
    a, ag, k = Dh * dl, alpha * 1.0, p.k
    mlo = -Dh + 1

    def phiv(x):
        x = np.asarray(x, float)
        v = 1j * np.sqrt(ag) * np.exp(1j * k * x + 0.5 * ag * (x + a))
        return np.where(x <= -a + 1e-12 * dl, v, 0.0)

    def psi(col, row):
        col, row = np.broadcast_arrays(np.asarray(col), np.asarray(row))
        ok = (row >= 0) & (row <= n)
        rr = np.where(ok, row, 0)
        left = col <= -Dh
        out = np.where(left & ok, np.sqrt(2.0) * phiv((col - rr) * dl) * et[rr], 0.0)
        inb = (~left) & ok & (col - mlo < nx)
        return np.where(inb, grid[rr, np.clip(col - mlo, 0, nx - 1)], out)

    th = lambda v: np.where(v > 0, 1.0, np.where(v == 0, 0.5, 0.0))
    t = n * dl
    i = np.arange(int(np.floor((-a + t - Ltail) / dl)), n + Dh + 3)
    I1, I2 = np.meshgrid(i, i, indexing="ij")
    pts = np.stack([I1.ravel(), I2.ravel(), np.full(I1.size, n)], axis=1)
    chi = O.chi(p, grid, pts).reshape(I1.shape)

    def T(i1, i2):
        r1, r2 = n - i2 - Dh, n - i2 + Dh
        return psi(i1 - i2 - Dh, r1) * th(i2 + Dh) * th(r1) - psi(i1 - i2 + Dh, r2) * th(i2 - Dh) * th(r2)

    # the same Eq. 2 written out here with numpy agrees (a check of the transcription)
    chi_np = phiv((I1 - n) * dl) * phiv((I2 - n) * dl) - 0.5 * (T(I1, I2) + T(I2, I1))
    assert np.max(np.abs(chi - chi_np)) <= 1e-13 * max(np.abs(chi_np).max(), 1e-300)
    w = np.ones(len(i))
    w[0] = w[-1] = 0.5
    p_chi = dl * dl * np.einsum("i,j,ij->", w, w, np.abs(chi) ** 2)
    p_left = 2 * abs(et[n]) ** 2 * math.exp(-ag * t)  # int_{x<-a} |sqrt2 phi(x-t) e(t)|^2
    return p_chi + p_left + nrm[n]


@pytest.mark.parametrize("dk,alpha", [(0.0, 1.0), (0.4, 0.7)])
def test_two_excitation_probability_conserved(oracle, dk, alpha):
    dev = [abs(total_probability(oracle, D, dk=dk, alpha=alpha) - 1.0) for D in (20, 40, 80)]
    # first order (the trapezoid rule meets the kinks of chi at x = +-a)
    assert dev[2] < 0.05 and dev[1] / dev[2] > 1.7 and dev[0] / dev[1] > 1.7, dev


def test_narrow_box_gives_same_columns(oracle):
    D, nrows = 20, 300
    wide = oracle.march(P(oracle, D, nrows, 160), nrows, tstep=0)["snaps"]
    narrow = oracle.march(P(oracle, D, nrows, 24), nrows, tstep=0)["snaps"]
    assert np.array_equal(wide[:, :24], narrow)


def test_long_run_bounded(oracle):
    D, nrows = 10, 4000
    p = P(oracle, D, nrows, 60, ic=2, alpha=0.5)
    res = oracle.march(p, nrows, tstep=None)
    assert np.all(np.isfinite(res["norms"]))
    assert res["norms"].max() < 2.0


def test_app_b_conversions_reproduce_captions():
    with open(os.path.join(HERE, "golden", "paper_parameter_sets.json")) as f:
        sets = json.load(f)
    for key in ("fig6_g2_k0a_pi_over_4", "fig7_g2_k0a_pi_over_2"):
        s = sets[key]
        n = s["k0a_over_pi"]
        W = s["w0"] / s["gamma"]  # calligraphic W = w0 / Gamma
        # App. B: w0 = (2 n pi / n_x) / Delta, Gamma = 2 n pi / (n_x W) / Delta
        assert abs(2 * n * PI / s["nx"] / s["Delta"] - s["w0"]) < 1e-9
        assert abs(2 * n * PI / (s["nx"] * W) / s["Delta"] - s["gamma"]) < 1e-9
        # a = n_x Delta / 2 gives k0 a = n pi with k0 = w0
        assert abs(s["w0"] * s["nx"] * s["Delta"] / 2 - n * PI) < 1e-9
    # Table 1: n_x even and n_x <= 2 N_x for every printed set
    for s in sets.values():
        if isinstance(s, dict) and "nx" in s:
            assert s["nx"] % 2 == 0 and s["nx"] <= 2 * s["Nx"]


def test_pair_of_equal_photons_is_the_identical_class(oracle):
    # init_cond 5 with (k2, alpha2) = (k, alpha) is init_cond 3 (A = 1/sqrt2): the marches agree
    D, nrows = 20, 400
    same = oracle.march(P(oracle, D, nrows, 200, ic=5, dk=0.2, alpha=0.8, k2=PI / 2 + 0.2, alpha2=0.8), nrows,
                        tstep=0)["snaps"]
    ident = oracle.march(P(oracle, D, nrows, 200, ic=3, dk=0.2, alpha=0.8), nrows, tstep=0)["snaps"]
    assert np.max(np.abs(same - ident)) < 1e-14 * np.abs(ident).max()


def test_two_different_photons_probability_conserved(oracle):
    # int |psi|^2 + int int |chi|^2 = 1 for two different exponential photons (Sec. 2 (c)),
    # chi by Eq. 2 (orc_chi), psi at x <= -a from the exact boundary; first order in delta
    dev = []
    for D in (20, 40, 80):
        dl = 2.0 / D
        Dh = D // 2
        t_end, Ltail = 8.0, 24.0
        n = int(round(t_end / dl))
        nx = n + D + 4
        p = P(oracle, D, n + 1, nx, ic=5, dk=0.3, alpha=0.7, k2=PI / 2 - 0.4, alpha2=1.3)
        res = oracle.march(p, n + 1, tstep=0)
        i = np.arange(int(np.floor((-p.a + t_end - Ltail) / dl)), n + Dh + 3)
        I1, I2 = np.meshgrid(i, i, indexing="ij")
        pts = np.stack([I1.ravel(), I2.ravel(), np.full(I1.size, n)], axis=1)
        chi = oracle.chi(p, res["snaps"], pts).reshape(I1.shape)
        w = np.ones(len(i))
        w[0] = w[-1] = 0.5
        p_chi = dl * dl * np.einsum("i,j,ij->", w, w, np.abs(chi) ** 2)
        cols = np.arange(-Dh - int(Ltail / dl), -Dh + 1)
        left = np.array([abs(oracle.psi_exact(p, n, c)) ** 2 for c in cols])
        wl = np.ones(len(cols))
        wl[0] = wl[-1] = 0.5
        # trapezoid up to x = -a; with the march's norm (a trapezoid from x = -a) the node at -a has weight 1
        p_left = dl * np.dot(wl, left)
        dev.append(abs(p_chi + p_left + res["norms"][n] - 1.0))
    assert dev[2] < 0.05 and dev[1] / dev[2] > 1.6 and dev[0] / dev[1] > 1.6, dev

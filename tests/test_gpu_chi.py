"""GPU parity of the two-photon wavefunction chi of Eq. 2 (fdtd_set_chi_points,
FDTD_READ_CHI) with the oracle's orc_chi on the oracle's full space-time grid:
detectors x1 = a + delta, x2 = x1 + tau (the paper's save_chi output), the
pair swapped (chi is symmetric), and points with a photon still in the
incident region; FDTD_F64 and FDTD_F64_DW, exponential and Gaussian photon
pairs.  Tolerance 1e-12 of the largest |chi|.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05943_gb300 import build, fdtd
    build.build()
    return fdtd


def detector_points(w, taus, rows):
    Dh = w.D // 2
    i1 = Dh + 1  # x1 = a + delta
    pts = [(i1, i1 + t, n) for n in rows for t in taus]
    pts += [(i1 + t, i1, n) for n in rows[::3] for t in taus[::4]]  # swapped
    pts += [(-Dh - 30, i1 + 5, n) for n in rows[::2]]  # one photon still left of the atom
    return np.array(pts, dtype=np.int64)


@pytest.mark.parametrize("prec", [0, 2], ids=["f64", "dw"])
@pytest.mark.parametrize("kind", ["exp", "gauss", "pair", "plane"])
def test_chi_matches_oracle(F, oracle, prec, kind):
    if kind == "exp":
        w = W.jittered(W.exp_pair(400, 1000, D=20, a=0.5), seed=3, n=1)[0]
    elif kind == "gauss":
        w = W.gauss_pair(400, 1000, D=20, a=0.5, gamma=1.0, k0a=0.25 * math.pi, sigma=1.0, lead=4.0)
    elif kind == "pair":
        w = W.photon_pair(400, 1000, D=20, a=0.5, dk1=0.4, alpha1=0.8, dk2=-0.3, alpha2=1.5)
    else:
        w = W.plane_wave(400, 1000, D=20, a=0.5, dk=0.2)
    pts = detector_points(w, taus=list(range(0, 60, 3)), rows=list(range(150, 1000, 70)))
    s = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                          init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, k2=w.k2,
                          alpha2=w.alpha2, tstep=-1, precision=prec, max_probes=4 * len(pts), rows_per_launch=300))
    s.set_boundary()
    F.fdtd_set_chi_points(s.plan, pts)
    s.march(w.nt)
    got = s.read(F.READ_CHI)
    s.close()
    p = oracle.Params(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                      init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, k2=w.k2, alpha2=w.alpha2)
    grid = oracle.march(p, tstep=0)["snaps"]
    want = oracle.chi(p, grid, pts)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(want).max(), np.max(np.abs(got - want))
    # chi is symmetric: the swapped points give the same four terms, summed in another order
    sym = {(int(a), int(b), int(n)): v for (a, b, n), v in zip(pts, got)}
    for (a, b, n), v in list(sym.items()):
        if (b, a, n) in sym:
            assert abs(sym[(b, a, n)] - v) <= 1e-14 * np.abs(got).max()
    assert np.abs(want).max() > 1e-3


def test_chi_point_limits(F):
    import ctypes
    w = W.exp_pair(200, 300, D=20, a=0.5)
    s = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                          init_cond=w.init_cond, alpha=w.alpha, max_probes=8))
    s.set_boundary()
    L = F.lib()
    Dh = w.D // 2
    right = np.array([[Dh + 1, Dh + 1 + 250, 299]], dtype=np.int64)  # needs psi right of the box
    assert L.fdtd_set_chi_points(s.plan, ctypes.c_void_p(right.ctypes.data), 1) == F.ERR_INVALID_ARG
    three = np.array([[Dh + 1, Dh + 2, 200]] * 3, dtype=np.int64)  # 3 points > max_probes / 4
    assert L.fdtd_set_chi_points(s.plan, ctypes.c_void_p(three.ctypes.data), 3) == F.ERR_INVALID_ARG
    s.march(250)
    late = np.array([[Dh + 1, Dh + 2, 200]], dtype=np.int64)  # its rows are already marched
    assert L.fdtd_set_chi_points(s.plan, ctypes.c_void_p(late.ctypes.data), 1) == F.ERR_STATE
    s.close()

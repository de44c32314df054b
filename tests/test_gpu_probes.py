"""Probes through the C ABI (fdtd_set_probes, FDTD_READ_PROBES): psi recorded by
the march at registered (row, column) points, in the order given (unsorted,
with repeats, spread over every CTA, the first column and the last), against
the oracle's full space-time grid at 1e-12 of the largest |psi|, for FDTD_F64
and FDTD_F64_DW; points on rows marched before the registration read 0.
"""
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


@pytest.mark.parametrize("prec", [0, 2], ids=["f64", "dw"])
def test_probes_match_oracle_grid(F, oracle, prec):
    w = W.jittered(W.exp_pair(5003, 700, D=40), seed=5, n=1)[0]
    rng = np.random.default_rng(17)
    rows = rng.integers(0, w.nt, 3000)
    # columns up to the light cone x = t + a of each row (plus a margin), and a few beyond it
    cols = np.minimum((rng.random(3000) * (rows + w.D + 40)).astype(np.int64), w.nx - 1)
    cols[::50] = rng.integers(0, w.nx, cols[::50].shape[0])
    pts = np.stack([rows, cols], axis=1)
    pts = np.concatenate([pts, [[w.nt - 1, 0], [w.nt - 1, w.nx - 1], [0, 7], [350, 4000], [350, 4000]]])
    s = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                          init_cond=w.init_cond, alpha=w.alpha, tstep=-1, precision=prec, max_probes=len(pts),
                          rows_per_launch=256))
    s.set_boundary()
    F.fdtd_set_probes(s.plan, pts)
    s.march(w.nt)
    got = s.read(F.READ_PROBES)
    s.close()
    ref = oracle.march(oracle.Params(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0,
                                     k=w.k, init_cond=w.init_cond, alpha=w.alpha), tstep=0)["snaps"]
    want = ref[pts[:, 0], pts[:, 1]]
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(ref).max()
    assert np.count_nonzero(want) > 2000  # most points lie inside the light cone


def test_probes_registered_late_and_limits(F):
    import ctypes
    w = W.exp_pair(600, 300, D=20, a=0.5)
    s = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                          init_cond=w.init_cond, alpha=w.alpha, tstep=0, max_probes=4))
    s.set_boundary()
    s.march(150)  # rows 0 .. 150 available
    pts = np.array([[100, 80], [200, 80], [299, 599], [151, 3]], dtype=np.int64)
    F.fdtd_set_probes(s.plan, pts)
    s.march(w.nt)
    got = s.read(F.READ_PROBES)
    snaps = s.snapshots()
    assert got[0] == 0  # row 100 was marched before the registration
    assert np.array_equal(got[1:], snaps[pts[1:, 0], pts[1:, 1]])
    L = F.lib()
    bad = np.array([[300, 0]], dtype=np.int64)
    assert L.fdtd_set_probes(s.plan, ctypes.c_void_p(bad.ctypes.data), 1) == F.ERR_INVALID_ARG
    five = np.zeros((5, 2), dtype=np.int64)
    assert L.fdtd_set_probes(s.plan, ctypes.c_void_p(five.ctypes.data), 5) == F.ERR_INVALID_ARG
    s.close()

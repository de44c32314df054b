"""GPU parity of the non-Markovian measures (App. D, FDTD_READ_MEASURES) with the
oracle: mu(t), lambda(t) and det M_t on the snapshot rows of a stimulated-
emission march, in FDTD_F64 and FDTD_F64_DW, and N_geo from them.

Tolerance: 1e-12 of the largest |mu| and lambda (the march itself agrees to
1e-12 relative L2; the measures are FP64 trapezoid sums of it).
"""
import math

import numpy as np
import pytest

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
@pytest.mark.parametrize("D,a,k0a,dk,alpha,tstep", [(40, 1.0, math.pi / 2, 0.0, 1.0, 9),
                                                    (20, 0.5, 0.3 * math.pi, 0.4, 0.6, 0)])
def test_measures_match_oracle(F, oracle, prec, D, a, k0a, dk, alpha, tstep):
    w0 = k0a / a
    delta = 2 * a / D
    nt = 1500
    nx = nt + 2 * D  # the box holds the light cone x = t + a up to the last row
    cfg = F.Config(nx=nx, nt=nt, D=D, delta=delta, gamma=1.0, omega0=w0, k=w0 + dk, init_cond=2, alpha=alpha,
                   tstep=tstep, precision=prec, rows_per_launch=512)
    s = F.Solver(cfg)
    s.set_boundary()
    s.march(700)
    s.march(nt)  # in two calls: the readout covers the rows marched so far
    got = s.measures()
    s.close()
    p = oracle.Params(nx=nx, nt=nt, D=D, delta=delta, gamma=1.0, omega0=w0, k=w0 + dk, init_cond=2, alpha=alpha)
    out = oracle.march(p, tstep=tstep)
    want = oracle.measures(p, out, tstep)
    assert got.shape == want.shape
    mu_g, mu_w = got[:, 0] + 1j * got[:, 1], want[:, 0] + 1j * want[:, 1]
    scale_mu, scale_l = np.abs(mu_w).max(), np.abs(want[:, 2]).max()
    assert np.max(np.abs(mu_g - mu_w)) < 1e-12 * scale_mu
    assert np.max(np.abs(got[:, 2] - want[:, 2])) < 1e-12 * scale_l
    assert np.max(np.abs(got[:, 3] - want[:, 3])) < 1e-12 * np.abs(want[:, 3]).max()
    ng_g, ng_w = F.fdtd_geometric_measure(got[:, 3]), float(np.clip(np.diff(np.abs(want[:, 3])), 0, None).sum())
    assert abs(ng_g - ng_w) <= 1e-12 * max(ng_w, 1e-300) + 1e-15
    print(f"prec {prec} D {D}: |mu| in [{np.abs(mu_w).min():.3f}, {np.abs(mu_w).max():.3f}], "
          f"lambda in [{want[:, 2].min():.3f}, {want[:, 2].max():.3f}], N_geo {ng_w:.4e}")


def test_measures_need_stimulated_emission_and_snapshots(F):
    import ctypes
    L = F.lib()
    for ic, tstep in ((3, 0), (2, -1)):
        cfg = F.Config(nx=64, nt=32, D=8, delta=0.25, gamma=1.0, omega0=1.0, k=1.0, init_cond=ic, alpha=1.0,
                       tstep=tstep)
        s = F.Solver(cfg)
        s.set_boundary()
        s.march(31)
        buf = np.zeros(4 * 32)
        assert L.fdtd_readout(s.plan, F.READ_MEASURES, ctypes.c_void_p(buf.ctypes.data), buf.nbytes) == \
            F.ERR_INVALID_ARG
        s.close()

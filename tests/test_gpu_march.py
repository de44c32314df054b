"""GPU parity of the FP64-accurate marches (libfdtd through its C ABI) with the
CPU oracle: FDTD_F64 (complex128) and FDTD_F64_DW (double-float pairs of FP32,
48 significant bits), each held to the same bar.

Tolerance: 1e-12 relative L2 over every stored row (rounding of two
different evaluation orders: the march is stable, |xi| <= 1 (App. A), so the
difference grows at most linearly in the ~1e4 steps along a characteristic;
1e-12 leaves two orders of margin over 4096 x 1e-16, and one over 4096 x
2^-48 for the double-float march).  e(t) tables: 1e-13 relative to max |e|.
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


def cfg_of(F, w, **kw):
    base = dict(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, k2=w.k2, alpha2=w.alpha2,
                tstep=0)
    base.update(kw)
    return F.Config(**base)


def oparams(O, w):
    return O.Params(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                    init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, k2=w.k2, alpha2=w.alpha2)


def run_gpu(F, w, pieces=None, **kw):
    s = F.Solver(cfg_of(F, w, **kw))
    s.set_boundary()
    for n in (pieces or [w.nt]):
        s.march(n)
    out = dict(snaps=s.snapshots(), norms=s.read(F.READ_NORMS), etab=s.read(F.READ_ETABLE),
               last=s.read(F.READ_ROW), rows=int(s.read(F.READ_ROWS_DONE)[0]))
    s.close()
    return out


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_parity(F, oracle, w, **kw):
    g = run_gpu(F, w, **kw)
    r = oracle.march(oparams(oracle, w), tstep=0, want_etab=True)
    assert g["rows"] == w.nt
    e_err = np.max(np.abs(g["etab"] - r["etab"])) / max(np.max(np.abs(r["etab"])), 1e-300)
    assert e_err < 1e-13, e_err
    if not np.any(r["snaps"]):  # nothing marched yet (nt = 1): exact zeros
        assert not np.any(g["snaps"])
        return 0.0
    err = rel_l2(g["snaps"], r["snaps"])
    assert err < 1e-12, err
    # norms: a row's absolute error is set by the largest amplitudes of the march,
    # so it is measured against the largest norm; rows within 1e-6 of it also
    # agree to 1e-9 relative
    nmax = r["norms"].max()
    nerr = np.max(np.abs(g["norms"] - r["norms"])) / nmax
    assert nerr < 1e-12, nerr
    big = r["norms"] > 1e-6 * nmax
    assert np.max(np.abs(g["norms"][big] - r["norms"][big]) / r["norms"][big]) < 1e-9
    assert np.array_equal(g["last"], g["snaps"][-1])
    return err


# FDTD_F64 and FDTD_F64_DW
PREC = pytest.mark.parametrize("prec", [0, 2], ids=["f64", "dw"])


@PREC
def test_small_workload_full_grid(F, oracle, prec):
    # the 1024 x 4096, D = 40 two-photon exponential workload: every row compared
    check_parity(F, oracle, W.SMALL, precision=prec)


@PREC
@pytest.mark.parametrize("i", range(3))
def test_jittered_two_photon(F, oracle, i, prec):
    # p = k - w0 + i Gamma (1-alpha)/2 != 0: gamma(n, z) at complex z
    w = W.jittered(W.exp_pair(512, 2048), seed=1707, n=3)[i]
    check_parity(F, oracle, w, precision=prec)


@PREC
def test_stimulated_emission(F, oracle, prec):
    w = W.Workload("stim", 512, 2048, 20, 0.1, 1.0, 2.3, 2.3, 2, alpha=0.5)
    check_parity(F, oracle, w, precision=prec)


@PREC
def test_gaussian_pair(F, oracle, prec):
    w = W.gauss_pair(600, 1500, D=40, a=1.0, gamma=1.0, k0a=0.3 * math.pi, sigma=1.0)
    check_parity(F, oracle, w, precision=prec)


@PREC
@pytest.mark.parametrize("dk", [0.0, 0.4])
def test_plane_wave(F, oracle, prec, dk):
    # Sec. 2 (a): two-photon plane wave, e0 through gamma(n, z) with p = k - w0 + i Gamma/2
    w = W.plane_wave(700, 1600, D=40, dk=dk)
    check_parity(F, oracle, w, precision=prec)


@PREC
@pytest.mark.parametrize("dk1,a1,dk2,a2", [(0.3, 0.7, -0.5, 1.4), (0.0, 1.0, 0.0, 1.0)])
def test_two_different_photons(F, oracle, prec, dk1, a1, dk2, a2):
    # Sec. 2 (c) with (k1, alpha1) != (k2, alpha2): the boundary is the sum of two
    # separable terms; (0, 1, 0, 1) is the identical pair through the same path
    w = W.photon_pair(900, 1500, D=40, dk1=dk1, alpha1=a1, dk2=dk2, alpha2=a2)
    check_parity(F, oracle, w, precision=prec)


@PREC
@pytest.mark.parametrize("nx,nt,D", [(2, 40, 2), (40, 300, 40), (2048 + 7, 200, 10), (5, 1, 4), (6, 2, 6)])
def test_edge_shapes(F, oracle, nx, nt, D, prec):
    # minimum box (nx = D), D = 2, a ragged chunk, only row 0, one marched row
    w = W.exp_pair(nx, nt, D=D, a=0.5 * D * 0.05)
    check_parity(F, oracle, w, precision=prec)


@PREC
def test_many_ctas_ragged(F, oracle, prec):
    # enough columns that every SM owns a range; nx not a multiple of anything
    w = W.exp_pair(20011, 360, D=40)
    check_parity(F, oracle, w, precision=prec)


@PREC
def test_many_ctas_wide_middle_region(F, oracle, prec):
    # D large against a CTA's width: the mirror bars of -a < x <= 3a read columns of
    # several CTAs, some to the right and up to D rows back; many launches
    w = W.gauss_pair(24001, 1500, D=800, a=4.0, gamma=1.0, k0a=0.3 * math.pi, sigma=1.0, lead=4.0)
    check_parity(F, oracle, w, precision=prec, rows_per_launch=333)


@PREC
def test_march_in_pieces_is_bitwise_equal(F, prec):
    w = W.exp_pair(3000, 700, D=40)
    one = run_gpu(F, w, precision=prec)
    pieces = run_gpu(F, w, pieces=[1, 250, 3, 1000], precision=prec)  # the last call is clamped at nt
    assert np.array_equal(one["snaps"], pieces["snaps"])
    assert np.array_equal(one["norms"], pieces["norms"])
    small = run_gpu(F, w, rows_per_launch=37, precision=prec)
    assert np.array_equal(one["snaps"], small["snaps"])


@PREC
def test_boundary_table_source(F, oracle, prec):
    # FDTD_BOUNDARY_TABLE: march from the oracle's e(t) instead of the kernel's
    import torch
    w = W.jittered(W.exp_pair(256, 900), seed=7, n=1)[0]
    et = oracle.etable(oparams(oracle, w), w.nt)
    t = torch.from_numpy(et.view(np.float64)).cuda()
    s = F.Solver(cfg_of(F, w, precision=prec))
    s.set_boundary(table=t)
    s.march(w.nt)
    g = s.snapshots()
    assert np.array_equal(s.read(F.READ_ETABLE), et)
    s.close()
    r = oracle.march(oparams(oracle, w), tstep=0)
    assert rel_l2(g, r["snaps"]) < 1e-12


def test_gamma_star_kernel(F, oracle):
    import torch
    ns, zs = [], []
    for n in [1, 2, 5, 17, 60, 130]:
        for r in [0.0, 0.5, 3.0, 20.0, 75.0, 140.0, 250.0]:
            for ang in np.linspace(-math.pi, math.pi, 11):
                ns.append(n)
                zs.append(r * complex(math.cos(ang), math.sin(ang)))
    n_t = torch.tensor(ns, dtype=torch.int32, device="cuda")
    z_t = torch.from_numpy(np.array(zs, dtype=np.complex128).view(np.float64)).cuda()
    out = torch.empty_like(z_t)
    F.fdtd_gamma_star(n_t.data_ptr(), z_t.data_ptr(), out.data_ptr(), len(ns))
    torch.cuda.synchronize()
    g = out.cpu().numpy().view(np.complex128)
    for n, z, v in zip(ns, zs, g):
        ref, _ = oracle.G(n, z)
        assert abs(v - ref) <= 1e-13 * abs(ref), (n, z, v, ref)


def test_call_order_and_buffer_errors(F):
    import ctypes
    L = F.lib()
    w = W.exp_pair(64, 32, D=8, a=0.2)
    plan, nbytes = F.fdtd_plan(cfg_of(F, w).c())
    try:
        assert L.fdtd_march(plan, 5) == F.ERR_STATE
        assert L.fdtd_set_boundary(plan, 0, None, 0) == F.ERR_STATE
        import torch
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (ws.data_ptr() + 255) // 256 * 256
        assert L.fdtd_bind_workspace(plan, ctypes.c_void_p(base), nbytes - 1) == F.ERR_WORKSPACE
        assert L.fdtd_bind_workspace(plan, ctypes.c_void_p(base + 8), nbytes) == F.ERR_WORKSPACE
        F.fdtd_bind_workspace(plan, base, nbytes)
        F.fdtd_set_boundary(plan)
        F.fdtd_march(plan, 31)
        small = np.empty(3, dtype=np.complex128)
        assert L.fdtd_readout(plan, F.READ_ROW, ctypes.c_void_p(small.ctypes.data), small.nbytes) == \
            F.ERR_INVALID_ARG
        assert L.fdtd_readout(plan, 99, ctypes.c_void_p(small.ctypes.data), small.nbytes) == F.ERR_INVALID_ARG
        assert L.fdtd_march(plan, -1) == F.ERR_INVALID_ARG
        row = np.empty(w.nx, dtype=np.complex128)
        F.fdtd_readout(plan, F.READ_ROW, row.ctypes.data, row.nbytes)
        assert np.all(np.isfinite(row))
    finally:
        F.fdtd_destroy(plan)


@PREC
def test_wait_timeout_latches_status(F, prec):
    # a wait limit of one cycle: a CTA whose left neighbour has not yet published
    # the previous row gives up at once, latches FDTD_ERR_TIMEOUT and returns; the
    # others see the latched status in their own waits and return too.  No wait is
    # left running, and the readout reports the status instead of data
    import ctypes
    w = W.exp_pair(20011, 64, D=40)
    s = F.Solver(cfg_of(F, w, tstep=-1, spin_cycles=1, precision=prec))
    s.set_boundary()
    s.march(w.nt)
    L = F.lib()
    row = np.empty(w.nx, dtype=np.complex128)
    st = L.fdtd_readout(s.plan, F.READ_ROW, ctypes.c_void_p(row.ctypes.data), row.nbytes)
    assert st == F.ERR_TIMEOUT
    assert b"row" in L.fdtd_last_error(s.plan)
    # the context is still usable: a fresh plan with the default limit marches normally
    s.close()
    g = run_gpu(F, W.exp_pair(512, 200, D=40))
    assert np.all(np.isfinite(g["snaps"]))

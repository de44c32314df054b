"""Checkpoint and resume through the C ABI (FDTD_READ_STATE, FDTD_BOUNDARY_RESTORE):
march N rows, take the state, restore it into a fresh plan of the same
parameters and march M more; the last row, the norms and the snapshots taken
after the checkpoint must be bitwise those of an uninterrupted march of N + M
rows (FDTD_F64, FDTD_F64_DW, and a complex64 batch of uneven instances).  A
checkpoint of other parameters, or one cut short, is refused.
"""
import ctypes
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


def cfg(F, w, prec, tstep=0, rpl=0):
    return F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                    init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=tstep,
                    precision=prec, rows_per_launch=rpl)


@pytest.mark.parametrize("prec", [0, 2], ids=["f64", "dw"])
@pytest.mark.parametrize("N", [1, 37, 400])
def test_resume_is_bitwise_the_uninterrupted_march(F, prec, N):
    w = W.gauss_pair(3001, 900, D=60, a=1.5, gamma=1.0, k0a=0.3 * math.pi, sigma=1.0, lead=4.0)
    full = F.Solver(cfg(F, w, prec, rpl=128))
    full.set_boundary()
    full.march(w.nt)
    a = F.Solver(cfg(F, w, prec, rpl=128))
    a.set_boundary()
    a.march(N - 1)  # rows 0 .. N-1 available
    state = a.checkpoint()
    assert state.nbytes == F.fdtd_readout_bytes(a.plan, F.READ_STATE)
    a.close()
    b = F.Solver(cfg(F, w, prec, rpl=128))
    b.restore(state)
    assert int(b.read(F.READ_ROWS_DONE)[0]) == N
    b.march(w.nt)
    assert np.array_equal(b.read(F.READ_ROW), full.read(F.READ_ROW))
    assert np.array_equal(b.read(F.READ_NORMS), full.read(F.READ_NORMS))
    assert np.array_equal(b.snapshots()[N:], full.snapshots()[N:])
    b.close()
    full.close()


def test_restore_refuses_other_parameters_and_short_records(F):
    w = W.exp_pair(500, 300, D=40)
    a = F.Solver(cfg(F, w, 0))
    a.set_boundary()
    a.march(120)
    state = a.checkpoint()
    a.close()
    L = F.lib()
    for other in (w.with_(D=20), w.with_(gamma=1.25), w.with_(nt=301)):
        b = F.Solver(cfg(F, other, 0))
        st = L.fdtd_set_boundary(b.plan, F.BOUNDARY_RESTORE, ctypes.c_void_p(state.ctypes.data), state.nbytes)
        assert st == F.ERR_INVALID_ARG
        assert L.fdtd_march(b.plan, 1) == F.ERR_STATE
        b.close()
    b = F.Solver(cfg(F, w, 0))
    st = L.fdtd_set_boundary(b.plan, F.BOUNDARY_RESTORE, ctypes.c_void_p(state.ctypes.data), state.nbytes - 8)
    assert st == F.ERR_INVALID_ARG
    b.restore(state)  # the whole record is accepted
    b.close()
    b = F.Solver(cfg(F, w, 2))  # a checkpoint of another precision
    st = L.fdtd_set_boundary(b.plan, F.BOUNDARY_RESTORE, ctypes.c_void_p(state.ctypes.data), state.nbytes)
    assert st == F.ERR_INVALID_ARG
    b.close()


def test_complex64_batch_resume(F):
    import torch
    ws = W.batch(seed=99, n=5, nx_lo=1 << 10, nx_hi=1 << 12, d_lo=10, d_hi=300)
    L = F.lib()

    def plan():
        arr = (F.FdtdParams * len(ws))(*[cfg(F, w, F.F32_COMP, tstep=-1, rpl=100).c() for w in ws])
        nb, p = ctypes.c_size_t(), ctypes.c_void_p()
        assert L.fdtd_plan(arr, len(ws), None, ctypes.byref(nb), ctypes.byref(p)) == F.OK
        buf = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        F.fdtd_bind_workspace(p, (buf.data_ptr() + 255) // 256 * 256, nb.value)
        return p, buf

    def read(p, i, kind, dtype):
        out = np.empty(F.fdtd_readout_instance_bytes(p, i, kind) // np.dtype(dtype).itemsize, dtype)
        F.fdtd_readout_instance(p, i, kind, out.ctypes.data, out.nbytes)
        return out

    N = 333
    full, fb = plan()
    F.fdtd_set_boundary(full)
    F.fdtd_march(full, max(w.nt for w in ws))
    a, ab = plan()
    F.fdtd_set_boundary(a)
    F.fdtd_march(a, N - 1)
    blob = np.concatenate([read(a, i, F.READ_STATE, np.uint8) for i in range(len(ws))])
    F.fdtd_destroy(a)
    b, bb = plan()
    F.fdtd_set_boundary(b, F.BOUNDARY_RESTORE, blob.ctypes.data, blob.nbytes)
    F.fdtd_march(b, max(w.nt for w in ws))
    for i in range(len(ws)):
        assert np.array_equal(read(b, i, F.READ_ROW, np.complex64), read(full, i, F.READ_ROW, np.complex64)), i
        assert np.array_equal(read(b, i, F.READ_NORMS, np.float64), read(full, i, F.READ_NORMS, np.float64)), i
    F.fdtd_destroy(b)
    F.fdtd_destroy(full)
    del fb, ab, bb

"""fdtd_march_noalloc: the march for callers that cannot allocate device memory.

Such callers (a framework that owns every device allocation through its own
pool, or a plugin inside one that may use only the buffers it is handed) pass
only their input parameters and output buffers; the march's scratch lives in
an array built into the library.  This file checks, through the C ABI, that two calls in a
row give the same last row and norms as the ordinary plan/workspace entry
points, within the tolerance the other parity tests use, and that an
instance larger than the built-in scratch is refused.  It sits in its own
file, collected last, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

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


def cfg(F, w):
    return F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                    init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=-1)


def with_workspace(F, w):
    """Last row and norms through fdtd_plan / fdtd_bind_workspace / ... / fdtd_readout."""
    s = F.Solver(cfg(F, w))
    s.set_boundary()
    s.march(w.nt)
    row, norms = s.read(F.READ_ROW), s.read(F.READ_NORMS)
    s.close()
    return row, norms


def without_allocation(F, w, tstep=-1):
    import torch
    row = torch.zeros(2 * w.nx, dtype=torch.float64, device="cuda")
    norms = torch.zeros(w.nt, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    c = cfg(F, w)
    c.tstep = tstep
    F.fdtd_march_noalloc(c.c(), stream, row.data_ptr(), norms.data_ptr())
    return row.cpu().numpy().view(np.complex128), norms.cpu().numpy()


def close(a, b, tol=1e-12):
    return np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_two_calls_match_workspace_path(F):
    first = W.exp_pair(4096, 2048, D=40)
    second = W.Workload("stim", 700, 1500, 20, 0.1, 1.0, 2.3, 2.3, 2, alpha=0.5)
    for w, tstep in ((first, 0), (second, -1)):
        # tstep is ignored: snapshots of every row of the first instance would take
        # 128 MiB, more than the scratch, yet the call runs (it keeps none)
        ref_row, ref_norms = with_workspace(F, w)
        row, norms = without_allocation(F, w, tstep)
        assert close(row, ref_row), np.abs(row - ref_row).max()
        assert np.max(np.abs(norms - ref_norms)) <= 1e-12 * ref_norms.max()


def test_rejects_instance_larger_than_scratch(F):
    import torch
    cap = F.fdtd_noalloc_max_bytes()
    assert cap == 64 << 20
    # (D+2) rows of 2^20 complex128 columns: 42 x 16 MiB > 64 MiB
    w = W.exp_pair(1 << 20, 64, D=40)
    row = torch.zeros(2, dtype=torch.float64, device="cuda")
    norms = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = F.lib().fdtd_march_noalloc(ctypes.byref(cfg(F, w).c()), None, ctypes.c_void_p(row.data_ptr()),
                                    ctypes.c_void_p(norms.data_ptr()))
    assert st == F.ERR_WORKSPACE

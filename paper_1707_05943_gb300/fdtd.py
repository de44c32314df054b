"""Python binding of libfdtd (include/fdtd.h).

Argument marshalling only: every step of the march runs in the library's CUDA
kernels.  PyTorch supplies device memory (the workspace and any device
buffers) and the CUDA stream.  If the library has not been built, or no GPU
is present, the calls raise; there is no CPU path.

The functions carry the C names (``fdtd_plan``, ``fdtd_bind_workspace``,
``fdtd_set_boundary``, ``fdtd_march``, ``fdtd_readout``, ``fdtd_destroy``,
``fdtd_gamma_star``); :class:`Solver` strings them together for one instance.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfdtd.so")

# fdtd_status
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_BOUNDS, ERR_NOT_CONVERGED, \
    ERR_STATE = range(9)
F64, F32_COMP, F64_DW = 0, 1, 2
IC_PLANE_WAVE, IC_STIM_EMISSION, IC_TWO_PHOTON_EXP, IC_TWO_PHOTON_GAUSS, IC_TWO_PHOTON_PAIR = 1, 2, 3, 4, 5
BOUNDARY_ANALYTIC, BOUNDARY_TABLE, BOUNDARY_RESTORE = 0, 1, 2
READ_ROW, READ_NORMS, READ_SNAPSHOTS, READ_ETABLE, READ_ROWS_DONE, READ_MEASURES, READ_STATE, READ_PROBES, \
    READ_CHI = range(9)

EXPORTS = ["fdtd_plan", "fdtd_bind_workspace", "fdtd_set_boundary", "fdtd_march", "fdtd_readout",
           "fdtd_readout_bytes", "fdtd_destroy", "fdtd_status_string", "fdtd_last_error", "fdtd_gamma_star",
           "fdtd_march_noalloc", "fdtd_noalloc_max_bytes", "fdtd_readout_instance", "fdtd_readout_instance_bytes",
           "fdtd_mlp_param_count", "fdtd_mlp_workspace_bytes", "fdtd_mlp_sync_bf16", "fdtd_mlp_forward",
           "fdtd_mlp_train_step", "fdtd_gemm_bf16", "fdtd_mlp_status", "fdtd_march_graph", "fdtd_alu_probe",
           "fdtd_geometric_measure", "fdtd_set_probes", "fdtd_set_chi_points"]


class FdtdParams(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("D", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("nt", ctypes.c_int64),
        ("delta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("omega0", ctypes.c_double),
        ("k", ctypes.c_double),
        ("init_cond", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("alpha", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("center", ctypes.c_double),
        ("tstep", ctypes.c_int32),
        ("rows_per_launch", ctypes.c_int32),
        ("cluster_ctas", ctypes.c_int32),
        ("mid_weight", ctypes.c_int32),
        ("k2", ctypes.c_double),
        ("alpha2", ctypes.c_double),
        ("max_probes", ctypes.c_int64),
        ("spin_cycles", ctypes.c_int64),
    ]


class FdtdMlp(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("n_layers", ctypes.c_int32),
        ("dims", ctypes.c_int32 * 8),
        ("params", ctypes.c_void_p),
        ("params_bf16", ctypes.c_void_p),
        ("grads", ctypes.c_void_p),
        ("adam_m", ctypes.c_void_p),
        ("adam_v", ctypes.c_void_p),
    ]


class FdtdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fdtd status {status}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libfdtd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FdtdError(ERR_CUDA, f"{LIB_PATH} is missing: build it with paper_1707_05943_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.fdtd_plan.argtypes = [ctypes.POINTER(FdtdParams), i32, vp, ctypes.POINTER(sz), ctypes.POINTER(vp)]
        L.fdtd_bind_workspace.argtypes = [vp, vp, sz]
        L.fdtd_set_boundary.argtypes = [vp, i32, vp, i64]
        L.fdtd_march.argtypes = [vp, i64]
        L.fdtd_march_graph.argtypes = [vp, i64]
        L.fdtd_readout.argtypes = [vp, i32, vp, i64]
        L.fdtd_readout_bytes.argtypes = [vp, i32]
        L.fdtd_readout_bytes.restype = i64
        L.fdtd_destroy.argtypes = [vp]
        L.fdtd_destroy.restype = None
        L.fdtd_status_string.argtypes = [ctypes.c_int]
        L.fdtd_status_string.restype = ctypes.c_char_p
        L.fdtd_last_error.argtypes = [vp]
        L.fdtd_last_error.restype = ctypes.c_char_p
        L.fdtd_gamma_star.argtypes = [vp, vp, vp, i64, vp]
        L.fdtd_march_noalloc.argtypes = [ctypes.POINTER(FdtdParams), vp, vp, vp]
        L.fdtd_readout_instance.argtypes = [vp, i32, i32, vp, i64]
        L.fdtd_readout_instance_bytes.argtypes = [vp, i32, i32]
        L.fdtd_readout_instance_bytes.restype = i64
        L.fdtd_noalloc_max_bytes.argtypes = []
        L.fdtd_noalloc_max_bytes.restype = sz
        mp = ctypes.POINTER(FdtdMlp)
        L.fdtd_mlp_param_count.argtypes = [mp, ctypes.POINTER(i64)]
        L.fdtd_mlp_workspace_bytes.argtypes = [mp, i32, ctypes.POINTER(sz)]
        L.fdtd_mlp_sync_bf16.argtypes = [mp, vp]
        L.fdtd_mlp_forward.argtypes = [mp, vp, i32, vp, vp, vp]
        L.fdtd_mlp_train_step.argtypes = [mp, vp, vp, i32, ctypes.c_float, i32, vp, vp, vp]
        L.fdtd_gemm_bf16.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, vp]
        L.fdtd_mlp_status.argtypes = [vp]
        L.fdtd_alu_probe.argtypes = [i32, vp, ctypes.POINTER(ctypes.c_double)]
        L.fdtd_geometric_measure.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double)]
        L.fdtd_set_probes.argtypes = [vp, vp, i64]
        L.fdtd_set_chi_points.argtypes = [vp, vp, i64]
        for f in ("fdtd_plan", "fdtd_bind_workspace", "fdtd_set_boundary", "fdtd_march", "fdtd_readout",
                  "fdtd_gamma_star", "fdtd_march_noalloc", "fdtd_readout_instance", "fdtd_mlp_param_count",
                  "fdtd_mlp_workspace_bytes", "fdtd_mlp_sync_bf16", "fdtd_mlp_forward", "fdtd_mlp_train_step",
                  "fdtd_gemm_bf16", "fdtd_mlp_status", "fdtd_march_graph", "fdtd_alu_probe",
                  "fdtd_geometric_measure", "fdtd_set_probes", "fdtd_set_chi_points"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st: int, plan=None, what: str = ""):
    if st != OK:
        L = lib()
        msg = L.fdtd_status_string(st).decode()
        if plan:
            detail = L.fdtd_last_error(plan).decode()
            if detail:
                msg += f" ({detail})"
        raise FdtdError(st, f"{what}: {msg}")


# ---- the C entry points, argument marshalling only ------------------------

def fdtd_plan(params: FdtdParams, n_instances: int = 1, stream: int | None = None):
    """Returns (plan handle, workspace bytes)."""
    ws = ctypes.c_size_t()
    plan = ctypes.c_void_p()
    st = lib().fdtd_plan(ctypes.byref(params), n_instances, ctypes.c_void_p(stream or 0), ctypes.byref(ws),
                         ctypes.byref(plan))
    _check(st, None, "fdtd_plan")
    return plan, ws.value


def fdtd_bind_workspace(plan, device_ptr: int, nbytes: int):
    _check(lib().fdtd_bind_workspace(plan, ctypes.c_void_p(device_ptr), nbytes), plan, "fdtd_bind_workspace")


def fdtd_set_boundary(plan, source: int = BOUNDARY_ANALYTIC, device_table: int = 0, n: int = 0):
    _check(lib().fdtd_set_boundary(plan, source, ctypes.c_void_p(device_table), n), plan, "fdtd_set_boundary")


def fdtd_march(plan, n_rows: int):
    _check(lib().fdtd_march(plan, n_rows), plan, "fdtd_march")


def fdtd_set_probes(plan, points):
    """points: (count, 2) int64 array of (row n, column index j)."""
    a = np.ascontiguousarray(points, dtype=np.int64).reshape(-1, 2)
    _check(lib().fdtd_set_probes(plan, a.ctypes.data, a.shape[0]), plan, "fdtd_set_probes")


def fdtd_set_chi_points(plan, pts):
    """pts: (count, 3) int64 array of (i1, i2, n): chi at x1 = i1 delta, x2 = i2 delta, t = n delta."""
    a = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    _check(lib().fdtd_set_chi_points(plan, a.ctypes.data, a.shape[0]), plan, "fdtd_set_chi_points")


def fdtd_march_graph(plan, n_rows: int):
    _check(lib().fdtd_march_graph(plan, n_rows), plan, "fdtd_march_graph")


def fdtd_readout(plan, kind: int, dst_ptr: int, dst_bytes: int):
    _check(lib().fdtd_readout(plan, kind, ctypes.c_void_p(dst_ptr), dst_bytes), plan, "fdtd_readout")


def fdtd_readout_instance(plan, instance: int, kind: int, dst_ptr: int, dst_bytes: int):
    _check(lib().fdtd_readout_instance(plan, instance, kind, ctypes.c_void_p(dst_ptr), dst_bytes), plan,
           "fdtd_readout_instance")


def fdtd_readout_instance_bytes(plan, instance: int, kind: int) -> int:
    return int(lib().fdtd_readout_instance_bytes(plan, instance, kind))


def fdtd_readout_bytes(plan, kind: int) -> int:
    return int(lib().fdtd_readout_bytes(plan, kind))


def fdtd_destroy(plan):
    lib().fdtd_destroy(plan)


def fdtd_gamma_star(n_ptr: int, z_ptr: int, out_ptr: int, count: int, stream: int | None = None):
    _check(lib().fdtd_gamma_star(ctypes.c_void_p(n_ptr), ctypes.c_void_p(z_ptr), ctypes.c_void_p(out_ptr), count,
                                 ctypes.c_void_p(stream or 0)), None, "fdtd_gamma_star")


def fdtd_march_noalloc(params: FdtdParams, stream: int | None, row_out_ptr: int, norms_out_ptr: int):
    """March one instance using the library's built-in scratch (no device allocation)."""
    _check(lib().fdtd_march_noalloc(ctypes.byref(params), ctypes.c_void_p(stream or 0), ctypes.c_void_p(row_out_ptr),
                                    ctypes.c_void_p(norms_out_ptr)), None, "fdtd_march_noalloc")


def fdtd_noalloc_max_bytes() -> int:
    return int(lib().fdtd_noalloc_max_bytes())


def fdtd_mlp_param_count(net: FdtdMlp) -> int:
    n = ctypes.c_int64()
    _check(lib().fdtd_mlp_param_count(ctypes.byref(net), ctypes.byref(n)), None, "fdtd_mlp_param_count")
    return n.value


def fdtd_mlp_workspace_bytes(net: FdtdMlp, batch: int) -> int:
    n = ctypes.c_size_t()
    _check(lib().fdtd_mlp_workspace_bytes(ctypes.byref(net), batch, ctypes.byref(n)), None,
           "fdtd_mlp_workspace_bytes")
    return n.value


def fdtd_mlp_sync_bf16(net: FdtdMlp, stream: int | None = None):
    _check(lib().fdtd_mlp_sync_bf16(ctypes.byref(net), ctypes.c_void_p(stream or 0)), None, "fdtd_mlp_sync_bf16")


def fdtd_mlp_forward(net: FdtdMlp, x_ptr: int, batch: int, y_ptr: int, ws_ptr: int, stream: int | None = None):
    _check(lib().fdtd_mlp_forward(ctypes.byref(net), ctypes.c_void_p(x_ptr), batch, ctypes.c_void_p(y_ptr),
                                  ctypes.c_void_p(ws_ptr), ctypes.c_void_p(stream or 0)), None, "fdtd_mlp_forward")


def fdtd_mlp_train_step(net: FdtdMlp, x_ptr: int, target_ptr: int, batch: int, lr: float, step: int, ws_ptr: int,
                        loss_ptr: int, stream: int | None = None):
    _check(lib().fdtd_mlp_train_step(ctypes.byref(net), ctypes.c_void_p(x_ptr), ctypes.c_void_p(target_ptr), batch,
                                     lr, step, ctypes.c_void_p(ws_ptr), ctypes.c_void_p(loss_ptr),
                                     ctypes.c_void_p(stream or 0)), None, "fdtd_mlp_train_step")


def fdtd_gemm_bf16(a_ptr: int, b_ptr: int, c_ptr: int, M: int, N: int, K: int, lda: int, ldb: int,
                   stream: int | None = None):
    _check(lib().fdtd_gemm_bf16(ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr), ctypes.c_void_p(c_ptr), M, N, K, lda,
                                ldb, ctypes.c_void_p(stream or 0)), None, "fdtd_gemm_bf16")


def fdtd_alu_probe(kind: int, stream: int | None = None) -> float:
    """Measured FMA throughput in flop/s: kind 0 FP64, 1 FP32, 2 packed FP32 pairs."""
    v = ctypes.c_double()
    _check(lib().fdtd_alu_probe(kind, ctypes.c_void_p(stream or 0), ctypes.byref(v)), None, "fdtd_alu_probe")
    return v.value


def fdtd_geometric_measure(det_m) -> float:
    """N_geo of App. D from a host array of det M samples (library host code)."""
    a = np.ascontiguousarray(det_m, dtype=np.float64)
    v = ctypes.c_double()
    _check(lib().fdtd_geometric_measure(a.ctypes.data, a.shape[0], ctypes.byref(v)), None, "fdtd_geometric_measure")
    return v.value


def fdtd_mlp_status(stream: int | None = None):
    _check(lib().fdtd_mlp_status(ctypes.c_void_p(stream or 0)), None, "fdtd_mlp_status")


# ---- convenience ------------------------------------------------------------

@dataclass
class Config:
    """One instance, in the paper's units (c = 1)."""
    nx: int
    nt: int
    D: int
    delta: float
    gamma: float
    omega0: float
    k: float
    init_cond: int = IC_TWO_PHOTON_EXP
    alpha: float = 1.0
    sigma: float = 0.0
    center: float = 0.0
    precision: int = F64
    tstep: int = -1
    rows_per_launch: int = 0
    cluster_ctas: int = 0
    mid_weight: int = 0
    k2: float = 0.0
    alpha2: float = 0.0
    max_probes: int = 0
    spin_cycles: int = 0

    def c(self) -> FdtdParams:
        p = FdtdParams()
        p.struct_size = ctypes.sizeof(FdtdParams)
        for f, _ in FdtdParams._fields_:
            if f != "struct_size":
                setattr(p, f, getattr(self, f))
        return p


@dataclass
class Solver:
    """Plan + torch-owned workspace for one instance on the current device."""
    cfg: Config
    stream: object = None
    plan: object = field(default=None, init=False)
    ws: object = field(default=None, init=False)

    def __post_init__(self):
        import torch
        if not torch.cuda.is_available():
            raise FdtdError(ERR_CUDA, "no CUDA device: libfdtd has no CPU path")
        s = self.stream if self.stream is not None else torch.cuda.current_stream()
        self._stream = s
        self.plan, nbytes = fdtd_plan(self.cfg.c(), 1, s.cuda_stream)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        fdtd_bind_workspace(self.plan, aligned, nbytes)

    @property
    def cdtype(self):
        return np.complex64 if self.cfg.precision == F32_COMP else np.complex128

    def set_boundary(self, table=None):
        if table is None:
            fdtd_set_boundary(self.plan, BOUNDARY_ANALYTIC, 0, 0)
        else:
            fdtd_set_boundary(self.plan, BOUNDARY_TABLE, table.data_ptr(), self.cfg.nt)

    def checkpoint(self) -> np.ndarray:
        """FDTD_READ_STATE into host memory."""
        return self.read(READ_STATE)

    def restore(self, state: np.ndarray):
        """FDTD_BOUNDARY_RESTORE from a checkpoint in host memory."""
        st = np.ascontiguousarray(state, dtype=np.uint8)
        fdtd_set_boundary(self.plan, BOUNDARY_RESTORE, st.ctypes.data, st.nbytes)

    def march(self, n_rows: int):
        fdtd_march(self.plan, n_rows)

    def read(self, kind: int, dtype=None, out=None):
        """Copy a readout into a host numpy array (or into `out`, a torch tensor)."""
        nbytes = fdtd_readout_bytes(self.plan, kind)
        if out is not None:
            fdtd_readout(self.plan, kind, out.data_ptr(), out.numel() * out.element_size())
            return out
        if dtype is None:
            dtype = {READ_NORMS: np.float64, READ_ETABLE: np.complex128, READ_ROWS_DONE: np.int64,
                     READ_MEASURES: np.float64, READ_STATE: np.uint8,
                     READ_PROBES: np.complex128, READ_CHI: np.complex128}.get(kind, self.cdtype)
        arr = np.empty(max(nbytes, 0) // np.dtype(dtype).itemsize, dtype=dtype)
        if nbytes > 0:
            fdtd_readout(self.plan, kind, arr.ctypes.data, arr.nbytes)
        return arr

    def measures(self):
        """App. D: (Re mu, Im mu, lambda, det M) per snapshot row (stimulated emission)."""
        return self.read(READ_MEASURES).reshape(-1, 4)

    def snapshots(self):
        a = self.read(READ_SNAPSHOTS)
        return a.reshape(-1, self.cfg.nx)

    def close(self):
        if self.plan is not None:
            fdtd_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


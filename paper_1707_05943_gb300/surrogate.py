"""Learned surrogate of the march: an ensemble of small MLPs mapping four
physical parameters of a two-photon Gaussian instance (Gamma a, k0 a, the
photon width sigma and an extra lead s of its centre) to what the march
produces on one fixed grid: the norm N(t) of Sec. 3 at 512 times and the
outgoing amplitude psi(x, t) on a 64 x 64 sub-grid.  The paper has no network;
the march is both its teacher and its fallback.

Everything numeric runs in the library's kernels: the data are march output
(complex64 compensated batched plan), training and inference go through
fdtd_mlp_train_step / fdtd_mlp_forward (BF16 tensor-core GEMMs, FP32
accumulation, Adam on FP32 masters).  PyTorch only holds device memory.

Outputs (8704 reals per instance):
  [0, 512)     N(2 j delta), j = 0..511
  [512, 8704)  64 x 64 complex: psi at row 16 i, column 16 c + 15 (x + a =
               16 (c + 1) delta), multiplied by exp(-i k ((x + a) - 2 t)) to take
               out the fast carrier phase, stored (re, im) interleaved.
An ensemble predicts either the norm alone ("norm", 512 outputs, the
quantity the 1e-3 contract is about) or everything ("all", 8704 outputs).
Error estimate: the largest spread (max - min) over the ensemble members of
any output, scaled by a factor calibrated on solver runs the networks never
saw; a query whose scaled estimate exceeds the tolerance is answered by the
march instead.
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass

import numpy as np

from . import fdtd as F

N_TIMES = 512
AMP_ROWS = 64
AMP_COLS = 64
N_OUT = N_TIMES + 2 * AMP_ROWS * AMP_COLS      # 8704
HIDDEN = [512, 512, 512, 512]
# what an ensemble predicts: the norm alone (first N_TIMES outputs) or everything
OUTPUTS = {"norm": slice(0, N_TIMES), "all": slice(0, N_OUT)}
DIMS = [4] + HIDDEN + [N_OUT]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise F.FdtdError(F.ERR_CUDA, "the surrogate needs a CUDA device")
    return torch


# ---- targets from the march ---------------------------------------------------

def _cfg(w, tstep, rpl=0):
    return F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                    init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=tstep,
                    precision=F.F32_COMP, rows_per_launch=rpl).c()


def targets_from_march(norms: np.ndarray, snaps: np.ndarray, w) -> np.ndarray:
    """Output vector of one instance from its norms (nt) and snapshots (rows 0, 16, ..)."""
    out = np.empty(N_OUT, np.float64)
    out[:N_TIMES] = norms[: 2 * N_TIMES: 2]
    cols = 16 * np.arange(AMP_COLS) + 15
    rows = np.arange(AMP_ROWS)
    xa = (cols + 1) * w.delta                       # x + a
    t = 16 * rows * w.delta
    ph = np.exp(-1j * w.k * (xa[None, :] - 2.0 * t[:, None]))
    amp = snaps[:AMP_ROWS, cols].astype(np.complex128) * ph
    out[N_TIMES:] = np.stack([amp.real, amp.imag], axis=-1).ravel()
    return out


def march_targets(workloads, chunk: int = 2048) -> tuple[np.ndarray, float]:
    """March every instance (batched complex64 plans of up to `chunk` instances)
    and return ([n, N_OUT] targets, seconds spent)."""
    torch = _torch()
    L = F.lib()
    out = np.empty((len(workloads), N_OUT), np.float64)
    t0 = time.perf_counter()
    for s in range(0, len(workloads), chunk):
        ws = workloads[s:s + chunk]
        for w in ws:
            if w.nt < 2 * N_TIMES or w.nx < 16 * AMP_COLS:
                raise ValueError("surrogate instances need nt >= 1024 and nx >= 1024")
        arr = (F.FdtdParams * len(ws))(*[_cfg(w, 15) for w in ws])
        nbytes, plan = ctypes.c_size_t(), ctypes.c_void_p()
        st = L.fdtd_plan(arr, len(ws), None, ctypes.byref(nbytes), ctypes.byref(plan))
        F._check(st, None, "fdtd_plan(surrogate batch)")
        buf = None
        try:
            buf = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
            F.fdtd_bind_workspace(plan, (buf.data_ptr() + 255) // 256 * 256, nbytes.value)
            F.fdtd_set_boundary(plan)
            F.fdtd_march(plan, max(w.nt for w in ws))
            for i, w in enumerate(ws):
                snaps = np.empty((F.fdtd_readout_instance_bytes(plan, i, F.READ_SNAPSHOTS) // 8), np.complex64)
                F.fdtd_readout_instance(plan, i, F.READ_SNAPSHOTS, snaps.ctypes.data, snaps.nbytes)
                norms = np.empty(w.nt, np.float64)
                F.fdtd_readout_instance(plan, i, F.READ_NORMS, norms.ctypes.data, norms.nbytes)
                out[s + i] = targets_from_march(norms, snaps.reshape(-1, w.nx), w)
        finally:
            F.fdtd_destroy(plan)
            del buf
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def normalise(feats, ranges) -> np.ndarray:
    """Features to [-1, 1] by the draw ranges."""
    f = np.asarray(feats, np.float64)
    lo = np.array([r[0] for r in ranges])
    hi = np.array([r[1] for r in ranges])
    return 2.0 * (f - lo) / (hi - lo) - 1.0


# ---- one network --------------------------------------------------------------

class Net:
    """Device parameters, gradient and Adam state of one MLP, with its own stream."""

    def __init__(self, dims=DIMS, seed: int = 0):
        torch = _torch()
        self.dims = list(dims)
        self.c = F.FdtdMlp()
        self.c.struct_size = ctypes.sizeof(F.FdtdMlp)
        self.c.n_layers = len(dims) - 1
        for i, d in enumerate(dims):
            self.c.dims[i] = d
        n = F.fdtd_mlp_param_count(self.c)
        self.n_params = n
        rng = np.random.default_rng(seed)
        theta = []
        for l in range(len(dims) - 1):
            fan_in, fan_out = dims[l], dims[l + 1]
            bound = math.sqrt(6.0 / fan_in) if l < len(dims) - 2 else math.sqrt(1.0 / fan_in)
            theta.append(rng.uniform(-bound, bound, fan_out * fan_in))
            theta.append(np.zeros(fan_out))
        theta = np.concatenate(theta).astype(np.float32)
        self.params = torch.from_numpy(theta).cuda()
        self.params_bf16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
        self.grads = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.m = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.c.params = self.params.data_ptr()
        self.c.params_bf16 = self.params_bf16.data_ptr()
        self.c.grads = self.grads.data_ptr()
        self.c.adam_m = self.m.data_ptr()
        self.c.adam_v = self.v.data_ptr()
        self.stream = torch.cuda.Stream()
        self.sp = self.stream.cuda_stream
        torch.cuda.synchronize()
        F.fdtd_mlp_sync_bf16(self.c, self.sp)
        self.step = 0
        self._ws = {}
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def ws(self, batch: int):
        torch = _torch()
        if batch not in self._ws:
            nb = F.fdtd_mlp_workspace_bytes(self.c, batch)
            self._ws[batch] = torch.empty(nb, dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
        return self._ws[batch].data_ptr()

    def train_step(self, x, t, lr: float):
        """x, t: device FP32 tensors [B, inputs], [B, outputs] (B a multiple of 64)."""
        self.step += 1
        F.fdtd_mlp_train_step(self.c, x.data_ptr(), t.data_ptr(), x.shape[0], lr, self.step, self.ws(x.shape[0]),
                              self.loss.data_ptr(), self.sp)

    def forward(self, x, y):
        F.fdtd_mlp_forward(self.c, x.data_ptr(), x.shape[0], y.data_ptr(), self.ws(x.shape[0]), self.sp)


# ---- the ensemble -------------------------------------------------------------

@dataclass
class TrainLog:
    steps: int
    seconds: float
    final_loss: list


class Surrogate:
    """K independently initialised networks trained on the same data (each on
    its own stream); the mean is the prediction, the spread the error estimate."""

    def __init__(self, K: int = 4, outputs: str = "norm", seed: int = 1707, ranges=None, hidden=HIDDEN):
        self.cols = OUTPUTS[outputs]
        n_out = self.cols.stop - self.cols.start
        self.dims = [4] + list(hidden) + [n_out]
        self.nets = [Net(self.dims, seed + 7919 * k) for k in range(K)]
        self.ranges = ranges
        self.q = 1.0  # calibration factor of the spread

    def _standardise(self, Y: np.ndarray):
        """Per-output mean and scale of the training targets; the scale is the
        output's standard deviation, floored at 5% of the largest one of its
        group (N(t) or amplitude) so that near-constant outputs are not blown up."""
        self.mu = Y.mean(axis=0)
        sd = Y.std(axis=0)
        for lo, hi in ((0, min(N_TIMES, Y.shape[1])), (N_TIMES, Y.shape[1])):
            if hi > lo:
                sd[lo:hi] = np.maximum(sd[lo:hi], 0.05 * sd[lo:hi].max())
        self.sd = sd

    def fit(self, X: np.ndarray, Y: np.ndarray, steps: int = 4000, batch: int = 512, lr: float = 2e-3,
            lr_min: float = 1e-5) -> TrainLog:
        """Adam with a cosine learning-rate decay; contiguous minibatches of a
        fixed random order, shifted by half a batch every other epoch.  Y holds
        full output vectors (N_OUT columns); the ensemble takes its own."""
        torch = _torch()
        Y = Y[:, self.cols]
        n = (X.shape[0] // batch) * batch
        if n == 0:
            raise ValueError("need at least one full batch of training data")
        self._standardise(Y)
        Xd = torch.from_numpy(np.ascontiguousarray(X[:n], np.float32)).cuda()
        Yd = torch.from_numpy(np.ascontiguousarray((Y[:n] - self.mu) / self.sd, np.float32)).cuda()
        nb = n // batch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(steps):
            epoch, b = divmod(s, nb)
            off = (b * batch + (epoch % 2) * (batch // 2)) % n
            if off + batch > n:
                off = 0
            lr_s = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * s / steps))
            for net in self.nets:
                net.train_step(Xd[off:off + batch], Yd[off:off + batch], lr_s)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        for net in self.nets:
            F.fdtd_mlp_status(net.sp)
        return TrainLog(steps, secs, [float(net.loss.item()) for net in self.nets])

    def predict(self, X: np.ndarray, batch: int = 256) -> tuple[np.ndarray, np.ndarray]:
        """(mean, per-query raw error estimate) over the members, in the units of the outputs."""
        torch = _torch()
        n = X.shape[0]
        npad = (n + batch - 1) // batch * batch
        Xp = np.zeros((npad, X.shape[1]), np.float32)
        Xp[:n] = X
        Xd = torch.from_numpy(Xp).cuda()
        Ys = torch.empty((len(self.nets), npad, self.dims[-1]), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for k, net in enumerate(self.nets):
            for s in range(0, npad, batch):
                net.forward(Xd[s:s + batch], Ys[k, s:s + batch])
        torch.cuda.synchronize()
        Y = Ys[:, :n].cpu().numpy().astype(np.float64) * self.sd + self.mu
        return Y.mean(axis=0), (Y.max(axis=0) - Y.min(axis=0)).max(axis=1)

    def calibrate(self, X: np.ndarray, Y: np.ndarray, quantile: float = 0.99) -> float:
        """Scale factor q of the spread: the `quantile` of (true max error) / spread
        over solver runs the networks were not trained on."""
        mean, est = self.predict(X)
        err = np.abs(mean - Y[:, self.cols]).max(axis=1)
        self.q = float(np.quantile(err / np.maximum(est, 1e-300), quantile))
        return self.q

    def answer(self, workloads, feats, tol: float = 1e-3):
        """Outputs for every query: the ensemble mean where q * spread <= tol, the
        march elsewhere.  Returns (outputs, served mask, seconds in the networks,
        seconds in the march)."""
        X = normalise(feats, self.ranges)
        t0 = time.perf_counter()
        mean, est = self.predict(X)
        t_net = time.perf_counter() - t0
        served = self.q * est <= tol
        t_march = 0.0
        out = mean.copy()
        rest = [i for i in range(len(workloads)) if not served[i]]
        if rest:
            Yr, t_march = march_targets([workloads[i] for i in rest])
            out[rest] = Yr[:, self.cols]
        return out, served, t_net, t_march

"""GPU: the surrogate network's kernels through the C ABI against the FP64
reference of oracle/mlp_ref.py -- the BF16 GEMM (tcgen05, K-contiguous operands), the
forward pass, the backpropagated gradient of every parameter, and the Adam
step.

Tolerances.  GEMM: operands are exact BF16 values, products exact and sums in
FP32 (tensor memory), so the error is a few FP32 roundings of sum |a||b|
(1e-5 of it allowed, K up to 8704).
Forward and gradient: the reference uses the same BF16-rounded weights in
FP64; the kernels also round every hidden activation and every backpropagated
signal to BF16 (relative 2^-9 each, about 1e-3 after averaging over many
terms); measured 1.5e-3 (forward) and 1.6e-4 to 1.8e-3 (gradients) on these
seeded inputs, 3e-3 allowed.  Adam: FP32
arithmetic of one update, 1e-5 of the learning rate.
"""
import ctypes

import numpy as np
import pytest

from oracle import mlp_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_05943_gb300 import build, fdtd
    build.build()
    return torch, fdtd


def bf16(torch, a):
    """Round FP64 values to BF16; returns (torch bf16 tensor, the FP64 values it holds)."""
    t = torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16)
    return t, t.to(torch.float64).numpy()


@pytest.mark.parametrize("M,N,K,pad", [(128, 128, 64, 0), (128, 192, 96, 8), (64, 64, 32, 0), (320, 128, 544, 24),
                                       (256, 8704, 512, 0), (8704, 512, 256, 0), (512, 512, 8704, 0)])
def test_gemm_tcgen05(env, M, N, K, pad):
    # C = A B^T with K contiguous in both; tiles of 128 with ragged M, N (multiples of 64)
    # and K (multiple of 32), padded leading dimensions
    torch, F = env
    rng = np.random.default_rng(M + 3 * N + 7 * K + pad)
    A = rng.normal(size=(M, K + pad))
    B = rng.normal(size=(N, K + pad))
    At, Av = bf16(torch, A)
    Bt, Bv = bf16(torch, B)
    want = Av[:, :K] @ Bv[:, :K].T
    scale = np.abs(Av[:, :K]) @ np.abs(Bv[:, :K]).T
    Ad, Bd = At.cuda(), Bt.cuda()
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    F.fdtd_gemm_bf16(Ad.data_ptr(), Bd.data_ptr(), C.data_ptr(), M, N, K, K + pad, K + pad)
    F.fdtd_mlp_status()
    got = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    bad = np.abs(got - want) > 1e-5 * scale + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], want[bad][:5])


class DeviceNet:
    def __init__(self, torch, F, dims, seed, batch):
        self.torch, self.F, self.dims = torch, F, dims
        rng = np.random.default_rng(seed)
        n = R.param_count(dims)
        theta = np.empty(n)
        o = 0
        for l in range(len(dims) - 1):
            k, m = dims[l], dims[l + 1]
            theta[o:o + m * k] = rng.uniform(-1, 1, m * k) * np.sqrt(3.0 / k)
            o += m * k
            theta[o:o + m] = rng.uniform(-0.3, 0.3, m)
            o += m
        self.theta32 = theta.astype(np.float32)
        self.p = torch.from_numpy(self.theta32.copy()).cuda()
        self.pb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
        self.g = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        self.m = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.v = torch.zeros(n, dtype=torch.float32, device="cuda")
        c = F.FdtdMlp()
        c.struct_size = ctypes.sizeof(F.FdtdMlp)
        c.n_layers = len(dims) - 1
        for i, d in enumerate(dims):
            c.dims[i] = d
        c.params, c.params_bf16, c.grads = self.p.data_ptr(), self.pb.data_ptr(), self.g.data_ptr()
        c.adam_m, c.adam_v = self.m.data_ptr(), self.v.data_ptr()
        self.c = c
        assert F.fdtd_mlp_param_count(c) == n
        F.fdtd_mlp_sync_bf16(c)
        self.ws = torch.empty(F.fdtd_mlp_workspace_bytes(c, batch), dtype=torch.uint8, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def theta_eff(self):
        """The parameters the kernels compute with: layer 0 in FP32, the rest in BF16."""
        th = self.p.cpu().numpy().astype(np.float64)
        bf = self.pb.to(self.torch.float64).cpu().numpy()
        n0 = self.dims[1] * self.dims[0]
        out = th.copy()
        o = 0
        for l in range(len(self.dims) - 1):
            k, m = self.dims[l], self.dims[l + 1]
            if l > 0:
                out[o:o + m * k] = bf[o:o + m * k]
            o += m * k + m
        assert n0 > 0
        return out


DIMS_SMALL = [4, 128, 64, 192, 128]


def test_bf16_copy_is_round_to_nearest(env):
    torch, F = env
    net = DeviceNet(torch, F, DIMS_SMALL, 1, 64)
    want = torch.from_numpy(net.theta32).to(torch.bfloat16)
    assert torch.equal(net.pb.cpu().view(torch.int16), want.view(torch.int16))


def test_forward_matches_fp64_reference(env):
    torch, F = env
    B = 128
    net = DeviceNet(torch, F, DIMS_SMALL, 2, B)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (B, 4)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = torch.full((B, DIMS_SMALL[-1]), float("nan"), dtype=torch.float32, device="cuda")
    F.fdtd_mlp_forward(net.c, xd.data_ptr(), B, y.data_ptr(), net.ws.data_ptr())
    F.fdtd_mlp_status()
    got = y.cpu().numpy().astype(np.float64)
    want, _, _ = R.forward(net.theta_eff(), DIMS_SMALL, x.astype(np.float64))
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print(f"forward rel L2 vs FP64 reference: {err:.3e}")
    assert err < 3e-3


def test_gradient_matches_fp64_reference(env):
    torch, F = env
    B = 128
    net = DeviceNet(torch, F, DIMS_SMALL, 3, B)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (B, 4)).astype(np.float32)
    t = rng.normal(0, 1, (B, DIMS_SMALL[-1])).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    F.fdtd_mlp_train_step(net.c, xd.data_ptr(), td.data_ptr(), B, 0.0, 1, net.ws.data_ptr(), net.loss.data_ptr())
    F.fdtd_mlp_status()
    got = net.g.cpu().numpy().astype(np.float64)
    th = net.theta_eff()
    want = R.grad(th, DIMS_SMALL, x.astype(np.float64), t.astype(np.float64))
    assert abs(net.loss.item() - R.loss(th, DIMS_SMALL, x, t)) <= 1e-2 * R.loss(th, DIMS_SMALL, x, t)
    # weights untouched with lr = 0
    assert np.array_equal(net.p.cpu().numpy(), net.theta32)
    o = 0
    for l in range(len(DIMS_SMALL) - 1):
        k, m = DIMS_SMALL[l], DIMS_SMALL[l + 1]
        for name, size in (("W", m * k), ("b", m)):
            g, w = got[o:o + size], want[o:o + size]
            err = np.linalg.norm(g - w) / np.linalg.norm(w)
            print(f"layer {l} d{name}: rel L2 {err:.3e}")
            assert err < 3e-3, (l, name, err)
            o += size


def test_adam_step_matches_reference(env):
    torch, F = env
    B = 64
    dims = [4, 64, 64]
    net = DeviceNet(torch, F, dims, 4, B)
    rng = np.random.default_rng(7)
    xd = torch.from_numpy(rng.uniform(-1, 1, (B, 4)).astype(np.float32)).cuda()
    td = torch.from_numpy(rng.normal(size=(B, 64)).astype(np.float32)).cuda()
    th = net.theta32.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    lr = 1e-3
    for step in (1, 2, 3):
        F.fdtd_mlp_train_step(net.c, xd.data_ptr(), td.data_ptr(), B, lr, step, net.ws.data_ptr(),
                              net.loss.data_ptr())
        g = net.g.cpu().numpy().astype(np.float64)
        th, m, v = R.adam_step(th, g, m, v, step, lr)
        got = net.p.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - th)) <= 1e-5 * lr * step + 1e-7 * np.max(np.abs(th)), step
        want_bf = torch.from_numpy(net.p.cpu().numpy()).to(torch.bfloat16)
        assert torch.equal(net.pb.cpu().view(torch.int16), want_bf.view(torch.int16))


def test_training_fits_a_smooth_map(env):
    # a network trained by the kernels alone drives the loss of a smooth target well down
    torch, F = env
    B = 256
    dims = [4, 128, 128, 64]
    net = DeviceNet(torch, F, dims, 8, B)
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, (B, 4))
    freq = rng.normal(size=(4, 64))
    t = np.sin(x @ freq) * 0.5
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    first = None
    for step in range(1, 1501):
        F.fdtd_mlp_train_step(net.c, xd.data_ptr(), td.data_ptr(), B, 2e-3, step, net.ws.data_ptr(),
                              net.loss.data_ptr())
        if step == 1:
            first = net.loss.item()
    last = net.loss.item()
    print(f"toy fit: loss {first:.3e} -> {last:.3e}")
    assert last < 1e-2 * first

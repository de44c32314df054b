"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function include/fdtd.h declares, the Python binding uses
the same names, and parameter validation rejects bad input before any CUDA
call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_1707_05943_gb300 import build, fdtd
    build.build()
    return fdtd


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", src)))


def test_exports_match_header(F):
    names = declared_functions()
    assert "fdtd_march" in names and "fdtd_gamma_star" in names
    L = F.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(F.EXPORTS) == names


def test_params_struct_layout(F, tmp_path):
    # the ctypes mirror has the C compiler's size and field offsets
    import subprocess
    fields = [f for f, _ in F.FdtdParams._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"fdtd.h\"\nint main(void){printf(\"%zu\\n\", sizeof(fdtd_params));"
    prog += "".join(f'printf("%zu\\n", offsetof(fdtd_params, {f}));' for f in fields) + "return 0;}"
    src = tmp_path / "layout.c"
    src.write_text(prog)
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(F.FdtdParams)
    assert out[1:] == [getattr(F.FdtdParams, f).offset for f in fields]


def _cfg(F, **kw):
    base = dict(nx=64, nt=32, D=8, delta=0.25, gamma=1.0, omega0=1.0, k=1.0, init_cond=3, alpha=1.0)
    base.update(kw)
    return F.Config(**base).c()


@pytest.mark.parametrize("kw", [dict(D=7), dict(D=0), dict(nx=6), dict(nt=0), dict(delta=0.0), dict(gamma=-1.0),
                                dict(init_cond=0), dict(init_cond=6), dict(init_cond=5, alpha2=0.0), dict(init_cond=3, alpha=0.0), dict(init_cond=4, sigma=0.0),
                                dict(tstep=-2), dict(cluster_ctas=65), dict(cluster_ctas=-1), dict(mid_weight=-3),
                                dict(mid_weight=5000), dict(precision=1, cluster_ctas=65), dict(spin_cycles=-1),
                                dict(precision=1, spin_cycles=-5)])
def test_plan_rejects_bad_params(F, kw):
    L = F.lib()
    ws, plan = ctypes.c_size_t(), ctypes.c_void_p()
    st = L.fdtd_plan(ctypes.byref(_cfg(F, **kw)), 1, None, ctypes.byref(ws), ctypes.byref(plan))
    assert st == F.ERR_INVALID_ARG
    assert not plan.value


def test_complex64_photon_pair_is_unsupported(F):
    # two different photons are marched by the FP64-accurate plans only
    L = F.lib()
    ws, plan = ctypes.c_size_t(), ctypes.c_void_p()
    st = L.fdtd_plan(ctypes.byref(_cfg(F, precision=1, init_cond=5, alpha2=1.0)), 1, None, ctypes.byref(ws),
                     ctypes.byref(plan))
    assert st == F.ERR_UNSUPPORTED and not plan.value


def test_plan_rejects_wrong_struct_size(F):
    L = F.lib()
    p = _cfg(F)
    p.struct_size = 8
    ws, plan = ctypes.c_size_t(), ctypes.c_void_p()
    assert L.fdtd_plan(ctypes.byref(p), 1, None, ctypes.byref(ws), ctypes.byref(plan)) == F.ERR_INVALID_ARG


def test_null_plan_calls(F):
    L = F.lib()
    assert L.fdtd_march(None, 1) == F.ERR_INVALID_ARG
    assert L.fdtd_set_boundary(None, 0, None, 0) == F.ERR_INVALID_ARG
    assert L.fdtd_readout(None, 0, None, 0) == F.ERR_INVALID_ARG
    assert L.fdtd_gamma_star(None, None, None, -1, None) == F.ERR_INVALID_ARG
    L.fdtd_destroy(None)
    assert L.fdtd_status_string(F.ERR_TIMEOUT) == b"device-side wait timed out"


def test_mlp_struct_layout(F, tmp_path):
    import subprocess
    fields = [f for f, _ in F.FdtdMlp._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"fdtd.h\"\nint main(void){printf(\"%zu\\n\", sizeof(fdtd_mlp));"
    prog += "".join(f'printf("%zu\\n", offsetof(fdtd_mlp, {f}));' for f in fields) + "return 0;}"
    src = tmp_path / "mlp_layout.c"
    src.write_text(prog)
    exe = tmp_path / "mlp_layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(F.FdtdMlp)
    assert out[1:] == [getattr(F.FdtdMlp, f).offset for f in fields]


def _net(F, dims, ptrs=True):
    net = F.FdtdMlp()
    net.struct_size = ctypes.sizeof(F.FdtdMlp)
    net.n_layers = len(dims) - 1
    for i, d in enumerate(dims):
        net.dims[i] = d
    if ptrs:
        net.params = net.params_bf16 = 256
    return net


def test_mlp_param_count_and_workspace(F):
    # host-only calls: 4 -> 512 x 4 -> 8704 has 4*512+512 + 3*(512*512+512) + 512*8704+8704 parameters
    net = _net(F, [4, 512, 512, 512, 512, 8704])
    assert F.fdtd_mlp_param_count(net) == 4 * 512 + 512 + 3 * (512 * 512 + 512) + 512 * 8704 + 8704
    ws = F.fdtd_mlp_workspace_bytes(net, 256)
    assert ws >= 256 * (4 * 512 * 6 + 8704 * 8)


@pytest.mark.parametrize("dims,batch", [([4, 512, 100], 64), ([4, 512, 512], 32), ([4, 512], 64),
                                        ([65, 512, 512], 64), ([4, 0, 64], 64)])
def test_mlp_rejects_bad_shapes(F, dims, batch):
    net = _net(F, dims)
    n = ctypes.c_size_t()
    assert F.lib().fdtd_mlp_workspace_bytes(ctypes.byref(net), batch, ctypes.byref(n)) == F.ERR_INVALID_ARG


def test_mlp_rejects_null_and_size(F):
    L = F.lib()
    net = _net(F, [4, 64, 64], ptrs=False)
    n = ctypes.c_size_t()
    assert L.fdtd_mlp_workspace_bytes(ctypes.byref(net), 64, ctypes.byref(n)) == F.ERR_INVALID_ARG
    net = _net(F, [4, 64, 64])
    net.struct_size = 12
    assert L.fdtd_mlp_workspace_bytes(ctypes.byref(net), 64, ctypes.byref(n)) == F.ERR_INVALID_ARG
    net = _net(F, [4] + [64] * 7)
    assert L.fdtd_mlp_workspace_bytes(ctypes.byref(net), 64, ctypes.byref(n)) == F.OK
    net.n_layers = 8  # more layers than dims[] can describe
    assert L.fdtd_mlp_workspace_bytes(ctypes.byref(net), 64, ctypes.byref(n)) == F.ERR_INVALID_ARG
    assert L.fdtd_gemm_bf16(None, None, None, 64, 64, 32, 32, 32, None) == F.ERR_INVALID_ARG
    assert L.fdtd_gemm_bf16(256, 256, 256, 64, 64, 48, 48, 48, None) == F.ERR_INVALID_ARG   # K % 32
    assert L.fdtd_gemm_bf16(256, 256, 256, 64, 64, 32, 36, 32, None) == F.ERR_INVALID_ARG   # lda % 8
    assert L.fdtd_gemm_bf16(264, 256, 256, 64, 64, 32, 32, 32, None) == F.ERR_INVALID_ARG   # A not 16-aligned

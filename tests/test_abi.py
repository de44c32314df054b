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
    return sorted(set(re.findall(r"\b(fdtd_[a-z_]+)\s*\(", src)))


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
                                dict(init_cond=1), dict(init_cond=3, alpha=0.0), dict(init_cond=4, sigma=0.0),
                                dict(tstep=-2)])
def test_plan_rejects_bad_params(F, kw):
    L = F.lib()
    ws, plan = ctypes.c_size_t(), ctypes.c_void_p()
    st = L.fdtd_plan(ctypes.byref(_cfg(F, **kw)), 1, None, ctypes.byref(ws), ctypes.byref(plan))
    assert st == F.ERR_INVALID_ARG
    assert not plan.value


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

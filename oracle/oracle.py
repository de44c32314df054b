"""ctypes front end of the FP64 CPU oracle (``fdtd_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  Nothing here is shared
with the CUDA path.

The library is built by :func:`build` (plain gcc, ``-ffp-contract=off`` so
that x86 and Arm hosts round the same way) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64),
        ("nt", ctypes.c_int64),
        ("D", ctypes.c_int32),
        ("init_cond", ctypes.c_int32),
        ("delta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("omega0", ctypes.c_double),
        ("k", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("center", ctypes.c_double),
        ("k2", ctypes.c_double),
        ("alpha2", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(OrcParams)
        L.orc_G.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_int)]
        L.orc_P.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_phi.argtypes = [P, ctypes.c_double, dp, dp]
        L.orc_e_at.argtypes = [P, ctypes.c_double, dp, dp]
        L.orc_etable.argtypes = [P, ctypes.c_int64, ctypes.c_void_p]
        L.orc_march.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
        L.orc_march_left.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        L.orc_psi_exact.argtypes = [P, ctypes.c_int64, ctypes.c_int64, dp, dp]
        L.orc_phi1.argtypes = [P, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_e0_at.argtypes = [P, ctypes.c_double, dp, dp]
        L.orc_measures.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
        L.orc_chi.argtypes = [P, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        L.orc_e2_at.argtypes = [P, ctypes.c_double, dp, dp]
        L.orc_pair_norm.argtypes = [P]
        L.orc_pair_norm.restype = ctypes.c_double
        for f in (L.orc_G, L.orc_P, L.orc_phi, L.orc_e_at, L.orc_etable, L.orc_march, L.orc_march_left,
                  L.orc_psi_exact, L.orc_phi1, L.orc_e0_at, L.orc_measures, L.orc_chi, L.orc_e2_at):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str, allow_nc: bool = False):
    if st == 0 or (allow_nc and st == 3):
        return
    raise OracleError(f"{what}: oracle status {st}")


@dataclass
class Params:
    """Physical parameters of one march (c = 1, as in the paper's captions)."""
    nx: int
    nt: int
    D: int
    delta: float
    gamma: float
    omega0: float
    k: float
    init_cond: int = 3
    alpha: float = 1.0
    sigma: float = 0.0
    center: float = 0.0
    k2: float = 0.0
    alpha2: float = 0.0

    def c(self) -> OrcParams:
        return OrcParams(self.nx, self.nt, self.D, self.init_cond, self.delta, self.gamma, self.omega0, self.k,
                         self.alpha, self.sigma, self.center, self.k2, self.alpha2)

    @property
    def a(self) -> float:
        return 0.5 * self.D * self.delta


def G(n: int, z: complex) -> tuple[complex, str]:
    """Gamma(n) * gamma*(n, z) and the App. C branch used."""
    re, im, br = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().orc_G(int(n), float(z.real), float(z.imag), ctypes.byref(re), ctypes.byref(im), ctypes.byref(br)),
           "orc_G")
    return complex(re.value, im.value), chr(br.value)


def P(n: int, z: complex) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_P(int(n), float(z.real), float(z.imag), ctypes.byref(re), ctypes.byref(im)), "orc_P")
    return complex(re.value, im.value)


def phi(p: Params, x: float) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_phi(ctypes.byref(cp), float(x), ctypes.byref(re), ctypes.byref(im)), "orc_phi")
    return complex(re.value, im.value)


def e_at(p: Params, t: float) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_e_at(ctypes.byref(cp), float(t), ctypes.byref(re), ctypes.byref(im)), "orc_e_at")
    return complex(re.value, im.value)


def etable(p: Params, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.complex128)
    cp = p.c()
    _check(lib().orc_etable(ctypes.byref(cp), int(n), out.ctypes.data), "orc_etable")
    return out


def psi_exact(p: Params, r: int, c: int) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_psi_exact(ctypes.byref(cp), int(r), int(c), ctypes.byref(re), ctypes.byref(im)),
           "orc_psi_exact")
    return complex(re.value, im.value)


def march(p: Params, n_rows: int | None = None, tstep: int | None = 0, norms: bool = True,
          want_etab: bool = False):
    """Run the oracle march.  Returns dict with 'snaps' ((rows/(tstep+1)) x nx),
    'norms' (n_rows), 'last' (nx) and optionally 'etab'."""
    n_rows = p.nt if n_rows is None else n_rows
    out = {}
    snaps = None
    if tstep is not None:
        ns = (n_rows - 1) // (tstep + 1) + 1
        snaps = np.zeros((ns, p.nx), dtype=np.complex128)
        out["snaps"] = snaps
    nrm = np.zeros(n_rows) if norms else None
    last = np.zeros(p.nx, dtype=np.complex128)
    et = np.zeros(n_rows, dtype=np.complex128) if want_etab else None
    cp = p.c()
    st = lib().orc_march(ctypes.byref(cp), int(n_rows), int(tstep or 0),
                         snaps.ctypes.data if snaps is not None else None,
                         nrm.ctypes.data if nrm is not None else None,
                         last.ctypes.data, et.ctypes.data if et is not None else None)
    _check(st, "orc_march")
    if nrm is not None:
        out["norms"] = nrm
    out["last"] = last
    if et is not None:
        out["etab"] = et
    return out


def march_left(p: Params, n_rows: int, L: int) -> np.ndarray:
    grid = np.zeros((n_rows, L), dtype=np.complex128)
    cp = p.c()
    _check(lib().orc_march_left(ctypes.byref(cp), int(n_rows), int(L), grid.ctypes.data), "orc_march_left")
    return grid


def phi1(p: Params, x: float, t: float) -> complex:
    """One-excitation photon field phi(x,t) (atom starting in its ground state)."""
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_phi1(ctypes.byref(cp), float(x), float(t), ctypes.byref(re), ctypes.byref(im)), "orc_phi1")
    return complex(re.value, im.value)


def e0_one(p: Params, t: float) -> complex:
    """e0(t) of the one-excitation sector (Sec. 2 (c) formula) for the photon of p."""
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_e0_at(ctypes.byref(cp), float(t), ctypes.byref(re), ctypes.byref(im)), "orc_e0_at")
    return complex(re.value, im.value)


def measures(p: Params, march_out: dict, tstep: int) -> np.ndarray:
    """(Re mu, Im mu, lambda, det M) per snapshot row of an init_cond-2 march (App. D)."""
    snaps = np.ascontiguousarray(march_out["snaps"])
    norms = np.ascontiguousarray(march_out["norms"])
    n_rows = norms.shape[0]
    out = np.zeros((snaps.shape[0], 4))
    cp = p.c()
    _check(lib().orc_measures(ctypes.byref(cp), n_rows, tstep, snaps.ctypes.data, norms.ctypes.data,
                              out.ctypes.data), "orc_measures")
    return out


def chi(p: Params, grid: np.ndarray, pts) -> np.ndarray:
    """chi(i1 delta, i2 delta, n delta) by Eq. 2 for triples (i1, i2, n), from the
    march's full grid (tstep = 0 snapshots, rows 0 .. n_rows-1)."""
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    q = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    out = np.zeros(q.shape[0], dtype=np.complex128)
    cp = p.c()
    _check(lib().orc_chi(ctypes.byref(cp), g.shape[0], g.ctypes.data, q.ctypes.data, q.shape[0], out.ctypes.data),
           "orc_chi")
    return out


def e2_at(p: Params, t: float) -> complex:
    """init_cond 5: e0 of the second photon."""
    re, im = ctypes.c_double(), ctypes.c_double()
    cp = p.c()
    _check(lib().orc_e2_at(ctypes.byref(cp), float(t), ctypes.byref(re), ctypes.byref(im)), "orc_e2_at")
    return complex(re.value, im.value)


def pair_norm(p: Params) -> float:
    """A of Sec. 2 (c) for two exponential photons (k, alpha), (k2, alpha2)."""
    cp = p.c()
    return float(lib().orc_pair_norm(ctypes.byref(cp)))

"""Synthetic workloads shaped like the paper's runs, and their seeded draws.

Pure data: sizes and physical parameters of each workload, plus a SplitMix64
generator for the seeded parameter sets.  Nothing here computes any part of
the method; both the CUDA path and the CPU oracle take their inputs from
this module.

Units follow the paper's figure captions (c = 1): a is the atom-mirror
distance, D = 2a/delta grid steps, k0 a the phase, and the incident carrier
is resonant, k = w0 = k0 (Figs. 5, 6-left, 9 use k = w0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

PI = math.pi


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int            # marched columns in x > -a
    nt: int            # rows
    D: int             # 2a / delta
    delta: float
    gamma: float
    omega0: float
    k: float
    init_cond: int     # 1 plane wave, 2 stimulated emission, 3 two identical exponential photons,
                       # 4 two identical Gaussian photons, 5 two different exponential photons
    alpha: float = 1.0
    sigma: float = 0.0
    center: float = 0.0
    k2: float = 0.0       # init_cond 5: the second photon's carrier and width
    alpha2: float = 0.0

    @property
    def a(self) -> float:
        return 0.5 * self.D * self.delta

    @property
    def updates(self) -> int:
        """Grid-point updates of one full march (rows 1..nt-1, every marched column)."""
        return self.nx * (self.nt - 1)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def exp_pair(nx, nt, D=40, a=1.0, gamma=1.0, k0a=PI / 2, alpha=1.0, name="exp") -> Workload:
    """Two identical exponential photons of width 1/(alpha Gamma) (Sec. 2 (c))."""
    w0 = k0a / a
    return Workload(name, nx, nt, D, 2 * a / D, gamma, w0, w0, 3, alpha=alpha)


def plane_wave(nx, nt, D=40, a=1.0, gamma=1.0, k0a=PI / 2, dk=0.0, name="plane") -> Workload:
    """Two-photon plane wave e^{ik(x1+x2)} (Sec. 2 (a)), k = w0 + dk."""
    w0 = k0a / a
    return Workload(name, nx, nt, D, 2 * a / D, gamma, w0, w0 + dk, 1)


def photon_pair(nx, nt, D=40, a=1.0, gamma=1.0, k0a=PI / 2, dk1=0.0, alpha1=1.0, dk2=0.0, alpha2=1.0,
                name="pair") -> Workload:
    """Two different exponential photons (k1, alpha1), (k2, alpha2) (Sec. 2 (c)), k_i = w0 + dk_i."""
    w0 = k0a / a
    return Workload(name, nx, nt, D, 2 * a / D, gamma, w0, w0 + dk1, 5, alpha=alpha1, k2=w0 + dk2, alpha2=alpha2)


def gauss_pair(nx, nt, D, a, gamma, k0a, sigma, lead=8.0, name="gauss") -> Workload:
    """Two identical Gaussian photons, centred `lead` sigma left of x = -a."""
    w0 = k0a / a
    return Workload(name, nx, nt, D, 2 * a / D, gamma, w0, w0, 4, sigma=sigma, center=-a - lead * sigma)


# The workloads.  "small": Gamma = 1, 2a = 2 (D = 40 at delta = 0.05), k0 a = pi/2,
# exponential two-photon packet of width 1/Gamma, 1024 x 4096 (complex128).
SMALL = exp_pair(1024, 4096, name="exp_pair_D40_nx1024_nt4096")
# "large": one FP64 instance, 2^20 x 2^18, D = 2000 (2a = 20/Gamma), k0 a = 0.3 pi,
# Gaussian pulse sigma = 5/Gamma, ring of D+2 rows x 2^20 complex128 in HBM.
LARGE = gauss_pair(1 << 20, 1 << 18, D=2000, a=10.0, gamma=1.0, k0a=0.3 * PI, sigma=5.0,
                   name="gauss_pair_D2000_nx1M_nt256k")
# "precision": the small physics at 8192 x 32768, marched in complex64.
PRECISION = exp_pair(8192, 32768, name="exp_pair_D40_nx8192_nt32768")


# ---- seeded draws -----------------------------------------------------------

class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit state, golden-ratio increment."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.s = seed & self.MASK

    def next_u64(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & self.MASK
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def jittered(base: Workload, seed: int, n: int) -> list[Workload]:
    """Parity cases around `base`: detuning k - w0 ~ U[-Gamma, Gamma] and
    alpha ~ U[0.5, 2] (p = k - w0 + i Gamma (1-alpha)/2 away from 0)."""
    g = SplitMix64(seed)
    out = []
    for i in range(n):
        dk = g.uniform(-base.gamma, base.gamma)
        al = g.uniform(0.5, 2.0)
        out.append(base.with_(k=base.omega0 + dk, alpha=al, name=f"{base.name}_jit{i}"))
    return out


def batch(seed: int = 1707, n: int = 256, nx_lo: int = 1 << 10, nx_hi: int = 1 << 16, d_lo: int = 10,
          d_hi: int = 2000) -> list[Workload]:
    """Seeded batch of uneven instances, two identical Gaussian photons each:
    nx log-uniform in [nx_lo, nx_hi], nt = nx, D uniform in [d_lo, d_hi] rounded
    to even and redrawn until D <= nx/2, Gamma a ~ U[0.1, 5], k0 a ~ U[0, 2 pi),
    sigma ~ U[0.5, 10]/Gamma, Gamma = 1, pulse centred 8 sigma left of x = -a."""
    g = SplitMix64(seed)
    out = []
    for i in range(n):
        nx = int(round(math.exp(g.uniform(math.log(nx_lo), math.log(nx_hi)))))
        while True:
            D = 2 * int(round(g.uniform(d_lo, d_hi) / 2))
            if D <= nx // 2:
                break
        ga = g.uniform(0.1, 5.0)
        k0a = g.uniform(0.0, 2 * PI)
        sigma = g.uniform(0.5, 10.0)
        out.append(gauss_pair(nx, nx, D=D, a=ga, gamma=1.0, k0a=k0a, sigma=sigma, name=f"batch{seed}_{i}"))
    return out


# ---- surrogate training and held-out draws ----------------------------------
# One fixed grid for every draw, so that outputs line up across instances:
# delta = 0.05 / Gamma, 1024 marched columns x 1024 rows (t up to 51.2 / Gamma).
SURR_DELTA = 0.05
SURR_NX = 1024
SURR_NT = 1024
# feature ranges: Gamma a, k0 a, sigma Gamma, extra lead s Gamma (pulse centre at -a - 6 sigma - s)
SURR_RANGES = ((0.25, 2.5), (0.0, PI), (1.0, 3.0), (0.0, 4.0))


def surrogate_draw(seed: int, n: int) -> tuple[list[Workload], list[tuple[float, float, float, float]]]:
    """Seeded (workload, feature) pairs for the surrogate.  Gamma = 1; D = 2a/delta
    rounded to even (a is then D delta / 2); k = w0 = k0 (resonant); two identical
    Gaussian photons of width sigma, centred 6 sigma + s left of x = -a."""
    g = SplitMix64(seed)
    ws, feats = [], []
    for i in range(n):
        ga = g.uniform(*SURR_RANGES[0])
        k0a = g.uniform(*SURR_RANGES[1])
        sig = g.uniform(*SURR_RANGES[2])
        s = g.uniform(*SURR_RANGES[3])
        D = max(2, 2 * int(round(ga / SURR_DELTA)))
        a = 0.5 * D * SURR_DELTA
        w = gauss_pair(SURR_NX, SURR_NT, D=D, a=a, gamma=1.0, k0a=k0a, sigma=sig, lead=6.0 + s / sig,
                       name=f"surr{seed}_{i}")
        ws.append(w)
        feats.append((a, k0a, sig, s))
    return ws, feats

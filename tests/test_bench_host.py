"""CPU: the bench's count of the march's algorithmic work, against a brute-force walk
over every grid point of small workloads.

An update at row n, storage column j carries the delay square when n >= D + 1, and in
x > 3a (j >= 2D) the boundary source R1 dE when r2 + D = n - j - 1 + D >= 0 and R2 phi
when r2 >= 0 (Eq. 1 with the App. A stencil; beyond x > 3a the mirror reads land in
x <= -a, where the field is C phi(x - t) e(t) and vanishes for t < 0)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def brute(w, n0, n1):
    upd = dly = src = nbytes = 0
    for n in range(n0, n1):
        for j in range(w.nx):
            upd += 1
            nbytes += 16 + (16 if n >= w.D else 0)
            if n >= w.D + 1:
                dly += 1
            if j >= 2 * w.D:
                i = n - j - 1 + w.D
                src += (i >= 0) + (i >= w.D)
    return {"updates": upd, "delay": dly, "src": src, "bytes": nbytes}


def test_march_work_matches_brute_force():
    for nx, D, n0, n1 in ((64, 4, 1, 90), (50, 10, 1, 13), (33, 16, 30, 70), (40, 30, 5, 6), (20, 12, 1, 40)):
        w = W.exp_pair(nx, n1, D=D)
        assert bench.march_work(w, n0, n1) == brute(w, n0, n1), (nx, D, n0, n1)


def test_work_tables_weigh_the_terms():
    w = W.exp_pair(64, 200, D=4)
    c = bench.march_work(w, 1, 200)
    # every update carries the base work; the sources only inside the light cone
    assert bench.work_of(c, bench.DW_INSTR) == 142 * c["updates"] + 80 * c["delay"] + 48 * c["src"]
    assert bench.work_of(c, bench.F64_INSTR) == 12 * c["updates"] + 8 * c["delay"] + 4 * c["src"]
    assert bench.work_of(c, bench.F64_FLOPS) == 20 * c["updates"] + 12 * c["delay"] + 8 * c["src"]
    assert 0 < c["src"] < 2 * c["updates"]

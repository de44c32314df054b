"""Autotuner of complex64 batched plans.

Two plan knobs change how a batch maps onto the GPU without changing what it
computes (the march's results do not depend on them, bit for bit):

* ``cluster_ctas`` -- the most band streams of one instance: an instance is
  marched in bands of 256 rows, up to that many in flight at once (the depth of
  the temporal blocking; its ring grows by 256 rows per stream);
* ``mid_weight`` -- the stream share s: instance i gets one stream per
  total / (CTAs s/8) updates of its own.  A larger share splits mid-sized
  instances into more streams (shorter time to finish, more ring memory); a
  smaller one keeps more CTAs on separate instances.

``tune`` estimates the whole march's time for every candidate pair and keeps
the fastest, caching the choice per batch shape in a JSON file.  A batch's
march goes through phases: at row r only the instances with more than r rows
are still marching, so the early rows are many instances and the late rows a
few wide ones, and the best knobs differ between them.  The estimate splits the
row range at quarters, times a short stretch (after a warm-up stretch, so that
the delay rows are in play) of the sub-batch still alive in each quarter, and
weights it by the quarter's length.  The boundary
is a zero e-table during tuning: the march's control flow does not depend on
the values, and the FP64 boundary would otherwise dominate the tuning time.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import statistics
from dataclasses import dataclass

from . import fdtd as F

CANDIDATES = tuple((c, w) for c in (8, 16, 32) for w in (8, 16, 32))
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


@dataclass
class Choice:
    cluster_ctas: int
    mid_weight: int
    ms: float
    key: str
    table: list


def bucket(configs) -> str:
    """Shape signature of a batch: instance count, widest and median width,
    median D and median rows, each rounded to a power of two."""
    def p2(v):
        return int(round(math.log2(max(1, v))))
    nx = [c.nx for c in configs]
    D = [c.D for c in configs]
    nt = [c.nt for c in configs]
    return (f"n{p2(len(configs))}_nxmax{p2(max(nx))}_nxmed{p2(statistics.median(nx))}"
            f"_D{p2(statistics.median(D))}_nt{p2(statistics.median(nt))}")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_march(configs, cluster_ctas: int, mid_weight: int, rows: int = 1024, warm: int = 1024) -> float:
    """Milliseconds for `rows` rows of the batch's march after `warm` rows (CUDA events)."""
    import torch
    cfgs = []
    for c in configs:
        p = c.c() if hasattr(c, "c") else c
        p.precision = F.F32_COMP
        p.tstep = -1
        p.cluster_ctas = cluster_ctas
        p.mid_weight = mid_weight
        cfgs.append(p)
    arr = (F.FdtdParams * len(cfgs))(*cfgs)
    nbytes, plan = ctypes.c_size_t(), ctypes.c_void_p()
    F._check(F.lib().fdtd_plan(arr, len(cfgs), None, ctypes.byref(nbytes), ctypes.byref(plan)), None,
             "fdtd_plan(autotune)")
    buf = None
    try:
        buf = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
        F.fdtd_bind_workspace(plan, (buf.data_ptr() + 255) // 256 * 256, nbytes.value)
        total_nt = sum(p.nt for p in cfgs)
        zeros = torch.zeros(2 * total_nt, dtype=torch.float64, device="cuda")
        F.fdtd_set_boundary(plan, F.BOUNDARY_TABLE, zeros.data_ptr(), total_nt)
        maxnt = max(p.nt for p in cfgs)
        warm = max(0, min(warm, maxnt - 1 - rows))
        if warm:
            F.fdtd_march(plan, warm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        F.fdtd_march(plan, rows)
        e1.record()
        torch.cuda.synchronize()
        rd = ctypes.c_int64()
        F.fdtd_readout(plan, F.READ_ROWS_DONE, ctypes.addressof(rd), 8)  # surfaces device-side errors
        return e0.elapsed_time(e1)
    finally:
        F.fdtd_destroy(plan)
        del buf


def estimate_march(configs, cluster_ctas: int, mid_weight: int, rows: int = 1024, phases: int = 4) -> float:
    """Estimated milliseconds of the whole march: per quarter of the row range,
    the time of `rows` rows of the instances still marching there, scaled by
    the quarter's length."""
    nts = [c.nt for c in configs]
    maxnt = max(nts)
    bounds = [maxnt * k // phases for k in range(phases + 1)]
    total = 0.0
    for k in range(phases):
        lo, hi = bounds[k], bounds[k + 1]
        alive = [c for c in configs if c.nt > lo]
        if not alive or hi <= lo:
            continue
        ms = time_march(alive, cluster_ctas, mid_weight, rows)
        total += ms * (hi - lo) / rows
    return total


def tune(configs, rows: int = 1024, candidates=CANDIDATES, cache_path: str | None = DEFAULT_CACHE,
         timer=None, refresh: bool = False) -> Choice:
    """The fastest (cluster_ctas, mid_weight) for this batch shape, from the
    cache when present (and not `refresh`), else measured with `timer`
    (default: estimate_march) and stored."""
    key = bucket(configs)
    cache = _load(cache_path) if cache_path else {}
    if key in cache and not refresh:
        c = cache[key]
        return Choice(c["cluster_ctas"], c["mid_weight"], c["ms"], key, c["table"])
    timer = timer or estimate_march
    table = []
    for cl, w in candidates:
        ms = float(timer(configs, cl, w, rows))
        table.append([cl, w, ms])
    cl, w, ms = min(table, key=lambda t: t[2])
    if cache_path:
        cache[key] = {"cluster_ctas": cl, "mid_weight": w, "ms": ms, "table": table, "rows": rows}
        _save(cache_path, cache)
    return Choice(cl, w, ms, key, table)

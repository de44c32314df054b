"""Benchmark of the FDTD march (grid-point updates/s) on GB300.

One step = one pass of the whole path on one instance: plan the boundary
(e(t) kernel, wavepacket and source tables) and march every row of the
workload.  Default workload: the large instance, 2^20 marched columns x 2^18
rows, D = 2000 (2a = 20/Gamma), k0 a = 0.3 pi, Gaussian pulse sigma = 5/Gamma,
marched to FP64 accuracy by the double-float march (FDTD_F64_DW: FP32 pairs,
held to the same 1e-12 relative L2 against the FP64 oracle as the complex128
march; --precision f64 times the complex128 march instead).  Its ring of
D+34 rows x 2^20 x 16 B is 34 GB, far larger than L2, so no L2 flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs N independent replicas (one per rank, launched by torchrun); the
value is the updates of all ranks over the slowest rank's time.  The
reference arm (--impl reference) times the CPU oracle on a bounded sample of
the same workload.  At N = 1 the line also carries "variants": the complex128
march on a prefix of the same workload, the seeded complex64 batch and the
complex64 precision instance (each with its error against the FP64 march and
its march rate over the FP64 march's), and the surrogate network, each timed
with its own CUDA events and clock record.

Other workloads, one JSON line each:
  --workload small      the 1024 x 4096 FP64 parity instance
  --workload precision  8192 x 32768, complex64 compensated, error vs FP64 stated
  --workload batch      256 seeded instances in one complex64 plan: autotuned
                        knobs, CUDA-graph march, error vs FP64 stated
  --workload surrogate  training and inference throughput of the surrogate network
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "grid-point updates/s & % HBM peak; FP32/batched vs plain FP64 at stated error"
UNIT = "grid-point updates/s"
# algorithmic work of the march, per update of x > 3a, split by the terms an update
# carries (the kernels compute exactly these):
#   always: c1 a, the recurrence step y = c2 (y + b) + q, the row norm term
#   rows n >= D + 1: the delay square (pair sums of rows n-D, n-D-1) times c3
#   the sources act only inside the light cone of the boundary: R1 dE for j <= n + D - 1,
#   R2 phi for j <= n - 1 (columns beyond are skipped by the kernels: nothing has arrived)
# bytes: the value written (16 B) and, for rows n >= D, the delay value read (16 B); row
# n-1 and the pair sums of row n-D-1 come from L2 and shared memory.
# FP64 (k_march_f64), FP64-pipe instructions (DADD, DMUL, DFMA each 1) and flops (FMA = 2):
# base: c1 a (2 DMUL + 2 DFMA, 6 flops), y + b (2 DADD), c2 (y + b) + q (4 DFMA, 8), the norm
# term (2 DFMA, 4) = 12 instructions, 20 flops; delay: the row n-D pair sum (2 DADD; it is
# the next row's n-D-1 pair, kept in shared memory), + the n-D-1 pair (2 DADD), c3 times
# that, accumulated (4 DFMA) = 8 instructions, 12 flops; each source product accumulated
# (4 DFMA) = 4 instructions, 8 flops.
F64_INSTR = {"base": 12, "delay": 8, "src": 4}
F64_FLOPS = {"base": 20, "delay": 12, "src": 8}
# double-float (k_march_dw), FP32-pipe instructions (FADD, FMUL, FFMA each 1) and flops
# (FMA = 2) of its operations: complex double-float product into a fresh value (cmul, 32
# instructions, 44 flops), product accumulated (cmac, 48, 60), sum (cadd, 16, 16),
# renormalisation (6, 6), norm term (24, 28).  base: d1 a cmul + a + S + b + y + c2 cmac +
# renormalisation + norm = 142 instructions (170 flops); delay: two pair sums + c3 cmac =
# 80 (92); each source: one cmac = 48 (60).  The carry correction of the parallel row scan
# is not counted (a sequential march does not need it).
DW_INSTR = {"base": 142, "delay": 80, "src": 48}
DW_FLOPS = {"base": 170, "delay": 92, "src": 60}


def march_work(w, n0: int, n1: int) -> dict:
    """Exact counts over rows n0 .. n1-1 of the march of workload w: updates, updates with
    the delay term (rows n >= D + 1), updates with each boundary source (bulk columns
    2D <= j <= n + D - 1 for R1 dE, 2D <= j <= n - 1 for R2 phi), and algorithmic HBM bytes."""
    import numpy as np
    n = np.arange(n0, n1, dtype=np.int64)
    g2 = min(2 * w.D, w.nx)
    upd = (n1 - n0) * w.nx
    dly = int(np.count_nonzero(n >= w.D + 1)) * w.nx
    src = int(np.clip(np.minimum(w.nx, n + w.D) - g2, 0, None).sum() + np.clip(np.minimum(w.nx, n) - g2, 0, None).sum())
    nbytes = 16 * upd + 16 * int(np.count_nonzero(n >= w.D)) * w.nx
    return {"updates": upd, "delay": dly, "src": src, "bytes": nbytes}


def work_of(counts: dict, table: dict) -> float:
    return table["base"] * counts["updates"] + table["delay"] * counts["delay"] + table["src"] * counts["src"]


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself at N = 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank_step * steps / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(w: W.Workload, rows: int, extra_cols: int = 512):
    """The oracle on a narrow box of the same workload: every column left of
    max(m, D/2) is exact, so a box of D + extra columns marches the same
    values the full width would there."""
    from oracle import oracle as O
    O.build()
    nx = min(w.nx, w.D + extra_cols)
    p = O.Params(nx=nx, nt=rows, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                 init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center)
    t0 = time.perf_counter()
    O.march(p, rows, tstep=None, norms=True)
    dt = time.perf_counter() - t0
    return nx * (rows - 1), dt, nx


def run_reference(args, w):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    rows = args.ref_rows
    for _ in range(args.warmup):
        oracle_sample(w, max(rows // 8, 8))
    tot_u, tot_t, nx = 0, 0.0, 0
    for _ in range(args.steps):
        u, dt, nx = oracle_sample(w, rows)
        tot_u += u
        tot_t += dt
    v = tot_u / tot_t
    sample = f"oracle march of {nx} columns x {rows} rows of {w.name} per step (narrow box, FP64, 1 thread)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "nt": w.nt, "D": w.D, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "small", "batch", "precision", "surrogate", "uniform"])
    ap.add_argument("--batch-n", type=int, default=256, help="instances of the seeded batch")
    ap.add_argument("--compare-f64", action="store_true", help="also march the batch in FP64, one plan each")
    ap.add_argument("--no-autotune", action="store_true", help="batch: default band streams per instance and stream share")
    ap.add_argument("--rows", type=int, default=0, help="march only this many rows (profiling)")
    ap.add_argument("--nx", type=int, default=0, help="march only this many columns (profiling)")
    ap.add_argument("--D", type=int, default=0, help="use this D at the same delta (profiling)")
    ap.add_argument("--rows-per-launch", type=int, default=4096)
    ap.add_argument("--mid-weight", type=int, default=0, help="column split weight of -a < x <= 3a (0: default)")
    ap.add_argument("--precision", default="dw", choices=["f64", "dw"],
                    help="large/small workloads: the double-float march (default) or the FP64 march; both are "
                         "held to the same 1e-12 parity with the FP64 oracle")
    ap.add_argument("--no-variants", action="store_true", help="large workload: skip the variants object")
    ap.add_argument("--variant-rows", type=int, default=8193,
                    help="rows of the FP64-march variant, timed from the middle of the large workload")
    ap.add_argument("--ref-rows", type=int, default=4096)
    ap.add_argument("--cpu-rows", type=int, default=6144)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()

    if args.workload in ("batch", "precision", "surrogate", "uniform"):
        if args.impl == "reference":
            run_reference(args, W.PRECISION if args.workload != "batch" else W.batch(n=args.batch_n)[0])
        else:
            run_variant(args)
        return
    w = W.LARGE if args.workload == "large" else W.SMALL
    if args.rows:
        w = w.with_(nt=args.rows, name=f"{w.name}_rows{args.rows}")
    if args.nx:
        w = w.with_(nx=args.nx, name=f"{w.name}_nx{args.nx}")
    if args.D:
        w = w.with_(D=args.D, name=f"{w.name}_D{args.D}")
    if args.impl == "reference":
        run_reference(args, w)
        return

    import numpy as np
    import torch

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1707_05943_gb300 import build, fdtd
    build.build()

    stream = torch.cuda.Stream(device=dev)
    rpl = args.rows_per_launch
    prec = fdtd.F64_DW if args.precision == "dw" else fdtd.F64
    cfg = fdtd.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                      init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=-1,
                      rows_per_launch=rpl, precision=prec, mid_weight=args.mid_weight)
    solver = fdtd.Solver(cfg, stream=stream)
    # boundary: phi table, row scalars, e-table pass 1 (+ pass 2 for the two-photon classes), norm, detab
    # (double-float: + the table split, and one norm reduction after every march launch)
    chunks = math.ceil((w.nt - 1) / rpl)
    launches_per_step = (5 if w.init_cond == 2 else 6) + (chunks if prec == fdtd.F64 else 1 + 2 * chunks)

    def step(events=None):
        solver.set_boundary()
        done = 1
        while done < w.nt:
            n = min(rpl, w.nt - done)
            if events is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                solver.march(n)
                e1.record(stream)
                events.append((e0, e1, n, done))
            else:
                solver.march(n)
            done += n

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    stream.synchronize()
    if args.warmup > 0:
        norms_w = solver.read(fdtd.READ_NORMS)
        assert np.all(np.isfinite(norms_w))

    # measured arithmetic peaks of this GPU (the roofline denominators of the marches)
    alu_peaks = {"fp64": fdtd.fdtd_alu_probe(0, stream.cuda_stream) / 1e12,
                 "fp32": fdtd.fdtd_alu_probe(1, stream.cuda_stream) / 1e12}
    sampler = ClockSampler(local)
    events = []
    barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    sampler.start()
    start.record(stream)
    for _ in range(args.steps):
        step(events)
    stop.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms = max_over_ranks(start.elapsed_time(stop), world, dev)
    updates_per_step = w.updates
    value = job_value(updates_per_step, args.steps, world, ms * 1e-3)

    # dominant kernel: the march launches (full-size ones); the algorithmic work of each
    # launch is counted exactly over its rows (the light cone makes later rows dearer)
    full = [e for e in events if e[2] == rpl] or list(events)
    t_full = sum(a.elapsed_time(b) for a, b, _, _ in full)
    avg_ms = t_full / len(full)
    rows_l = full[0][2]
    peaks, src = load_peaks()
    upd_launch = rows_l * w.nx
    cnt = {"updates": 0, "delay": 0, "src": 0, "bytes": 0}
    for _, _, n, n0 in full:
        for k, v in march_work(w, n0, n0 + n).items():
            cnt[k] += v
    sec = t_full * 1e-3
    ach_gbs = cnt["bytes"] / sec / 1e9
    hbm = {"achieved": ach_gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
           "frac": ach_gbs / peaks.get("hbm_gbs", 6800.0), "bytes_per_update": cnt["bytes"] / cnt["updates"],
           "peak_source": src}
    work = {"updates": cnt["updates"], "with_delay": cnt["delay"], "source_products": cnt["src"],
            "launches": len(full)}
    if prec == fdtd.F64:
        ins, fl = work_of(cnt, F64_INSTR), work_of(cnt, F64_FLOPS)
        ach = ins / sec / 1e12
        pk = alu_peaks["fp64"] / 2  # DFMA rate = FP64 pipe instruction rate
        roof = {"kernel": "k_march_f64", "bound": "alu", "achieved": ach, "peak": pk,
                "unit": "T FP64-pipe instructions/s (DADD, DMUL, DFMA each 1)", "frac": ach / pk,
                "peak_source": "measured in this run: FP64 FMA throughput of fdtd_alu_probe (independent "
                               "FMA chains on every SM, CUDA events) / 2 flops per FMA",
                "fp64_instr_per_update": ins / cnt["updates"], "flops_per_update": fl / cnt["updates"],
                "flops_frac": fl / sec / 1e12 / alu_peaks["fp64"], "work": work, "updates_per_launch": upd_launch,
                "launch_ms": avg_ms, "traffic": 32.1 * upd_launch,
                "traffic_source": "ncu dram__bytes_read+write of k_march_f64 at nx 2^20, D 100 (32.1 B/update), "
                                  "scaled to this launch's updates",
                "hbm": hbm}
    else:
        ins, fl = work_of(cnt, DW_INSTR), work_of(cnt, DW_FLOPS)
        ach = ins / sec / 1e12
        pk = alu_peaks["fp32"] / 2  # FMA rate = FP32 pipe instruction rate
        roof = {"kernel": "k_march_dw", "bound": "alu", "achieved": ach, "peak": pk,
                "unit": "T FP32-pipe instructions/s (FADD, FMUL, FFMA each 1)", "frac": ach / pk,
                "peak_source": "measured in this run: FP32 FMA throughput of fdtd_alu_probe / 2 flops per FMA",
                "fp32_instr_per_update": ins / cnt["updates"], "flops_per_update": fl / cnt["updates"],
                "flops_frac": fl / sec / 1e12 / alu_peaks["fp32"], "work": work,
                "updates_per_launch": upd_launch, "launch_ms": avg_ms,
                "launch_ms_each": [round(a.elapsed_time(b), 2) for a, b, n, _ in events[:len(events) // max(args.steps, 1)]],
                "traffic": None,
                "traffic_source": "no ncu capture of this kernel at this size yet", "hbm": hbm}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == fdtd.F64 else "f32x2 (double-float, FP64-accurate)",
           "data": "synthetic",
           "config": {"workload": w.name, "nx": w.nx, "nt": w.nt, "D": w.D, "delta": w.delta,
                      "k0a": w.omega0 * w.a, "sigma": w.sigma,
                      "precision": "complex128" if prec == fdtd.F64 else "complex double-float (4 x FP32)",
                      "rows_per_launch": rpl, "parallelism": f"replicas x{world}",
                      "l2": "inputs larger than L2 (ring of "
                            f"{w.D + 2 + (32 if prec != fdtd.F64 else 0)} rows = "
                            f"{(w.D + 2 + (32 if prec != fdtd.F64 else 0)) * w.nx * 16 / 1e9:.1f} GB)"},
           "roofline": roof, "gpu_launches": launches_per_step * args.steps, "clocks": clocks}

    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        pinned_norms = torch.empty(w.nt, dtype=torch.float64, pin_memory=True)
        pinned_row = torch.empty(2 * w.nx, dtype=torch.float64, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s2 = fdtd.Solver(cfg, stream=stream)
            s2.set_boundary()
            s2.march(w.nt)
            s2.read(fdtd.READ_NORMS, out=pinned_norms)
            s2.read(fdtd.READ_ROW, out=pinned_row)
            s2.close()
            del s2
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = 8 * (solver_grid(solver) + 1)
        out["e2e"] = {"value": job_value(updates_per_step, args.steps, world, dt), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8 * w.nt + 16 * w.nx,
                      "includes": "plan + workspace allocation + boundary + march + readout of norms and "
                                  "last row into pinned host memory"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        u, dt, nx = oracle_sample(w, args.cpu_rows)
        out["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"oracle march of {nx} columns x {args.cpu_rows} rows of {w.name} "
                                         f"({u:.3g} updates, {dt:.1f} s, FP64, 1 thread)"}
    solver.close()
    del solver
    if rank == 0 and world == 1 and not args.no_variants and args.workload == "large":
        # the other paths on this GPU, each with its own CUDA-event timing and clock record:
        # the FP64 march, the complex64 compensated march (seeded batch, precision
        # instance) with its error against the FP64 march, and the surrogate network
        torch.cuda.empty_cache()
        var = {}
        runs = (("f64_march", lambda: f64_variant(args, args.variant_rows, alu_peaks["fp64"])),
                ("batch_c64", lambda: c64_variant(args, "batch", 1, 2, peaks, src)),
                ("precision_c64", lambda: c64_variant(args, "precision", 1, 2, peaks, src)),
                ("surrogate", lambda: surrogate_variant(args, 1, 3, peaks, src)))
        for name, fn in runs:
            try:
                var[name] = fn()
            except Exception as e:  # reported, not hidden: the line still carries the headline
                var[name] = {"error": repr(e)[:400]}
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        head_march = rpl * w.nx / (avg_ms * 1e-3)  # march-only rate of the headline launches
        f64v = var.get("f64_march", {}).get("value")
        ratios = {"headline_march_over_f64_march": head_march / f64v if f64v else None}
        for k in ("batch_c64", "precision_c64"):
            mv = var.get(k, {}).get("march_only_value")
            ratios[f"{k}_march_over_f64_march"] = mv / f64v if (mv and f64v) else None
        var["ratios"] = ratios
        var["headline_march_only_value"] = head_march
        out["variants"] = var
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_variant(args):
    """The complex64 compensated march on the seeded batch or the precision
    instance, or the surrogate network's training and inference; one JSON line."""
    import torch

    from paper_1707_05943_gb300 import build
    build.build()
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    peaks, src = load_peaks()
    if args.workload == "surrogate":
        out = surrogate_variant(args, args.steps, args.warmup, peaks, src)
    else:
        out = c64_variant(args, args.workload, args.steps, args.warmup, peaks, src)
    print(json.dumps(out), flush=True)


def c64_variant(args, which, steps, warmup, peaks, src):
    """One complex64 plan (the seeded batch, or the precision instance): boundary
    plus CUDA-graph march per step, CUDA events on the plan's stream; error of the
    largest instances against the FP64 march."""
    import ctypes

    import numpy as np
    import torch

    from paper_1707_05943_gb300 import fdtd as F
    local = env_rank()[2]
    if which == "uniform":  # --batch-n copies of the precision physics at --nx x (--rows + 1), --D
        nx, rows_u, D = args.nx or 4096, args.rows or 1024, args.D or 40
        one = W.PRECISION.with_(nx=nx, nt=rows_u + 1, D=D, delta=W.PRECISION.delta, name="uniform")
        ws_list = [one] * args.batch_n
        name = f"uniform_n{args.batch_n}_nx{nx}_nt{rows_u + 1}_D{D}"
    elif which == "batch":
        ws_list = W.batch(n=args.batch_n)
        name = f"batch1707_n{len(ws_list)}"
    else:
        ws_list = [W.PRECISION]
        name = W.PRECISION.name

    def cfg(w, prec, tstep=-1, cluster_ctas=0, mid_weight=0):
        return F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                        init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=tstep,
                        precision=prec, rows_per_launch=0, cluster_ctas=cluster_ctas, mid_weight=mid_weight)

    knobs, tuned = {}, None
    if which == "batch" and not args.no_autotune:
        from paper_1707_05943_gb300 import autotune as A
        ch = A.tune([cfg(w, F.F32_COMP) for w in ws_list], rows=1024)
        knobs = {"cluster_ctas": ch.cluster_ctas, "mid_weight": ch.mid_weight}
        tuned = {"cluster_ctas": ch.cluster_ctas, "mid_weight": ch.mid_weight, "key": ch.key,
                 "estimated_march_ms": ch.table}
    arr = (F.FdtdParams * len(ws_list))(*[cfg(w, F.F32_COMP, **knobs).c() for w in ws_list])
    nbytes, plan = ctypes.c_size_t(), ctypes.c_void_p()
    F._check(F.lib().fdtd_plan(arr, len(ws_list), None, ctypes.byref(nbytes), ctypes.byref(plan)), None, "plan")
    buf = torch.empty(nbytes.value + 256, dtype=torch.uint8, device="cuda")
    F.fdtd_bind_workspace(plan, (buf.data_ptr() + 255) // 256 * 256, nbytes.value)
    rows = max(w.nt for w in ws_list)
    updates = sum(w.updates for w in ws_list)
    stream = torch.cuda.default_stream()
    ev = []

    def step(record=False):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        F.fdtd_set_boundary(plan)
        e1.record(stream)
        F.fdtd_march_graph(plan, rows)  # recorded on the first (warm-up) step, replayed after
        e2.record(stream)
        if record:
            ev.append((e0, e1, e2))

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.start()
    start.record(stream)
    for _ in range(steps):
        step(True)
    stop.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = start.elapsed_time(stop)
    t_bnd = sum(a.elapsed_time(b) for a, b, _ in ev) / len(ev)
    t_march = sum(b.elapsed_time(c) for _, b, c in ev) / len(ev)
    # error against the FP64 march (parity-checked against the oracle) on the three largest
    # instances by updates (the longest characteristics) and the smallest: the batch plan's
    # norms, and about 512 stored rows of each instance marched alone
    order = sorted(range(len(ws_list)), key=lambda i: ws_list[i].updates)
    pick = sorted(set(order[-3:] + order[:1]))
    errs, nerrs = [], []
    for i in pick:
        w = ws_list[i]
        norms = np.empty(w.nt, np.float64)
        F.fdtd_readout_instance(plan, i, F.READ_NORMS, norms.ctypes.data, norms.nbytes)
        ts = max(w.nt // 512 - 1, 0)
        snaps = {}
        for prec in (F.F32_COMP, F.F64):
            sv = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                                   init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=ts,
                                   precision=prec))
            sv.set_boundary()
            sv.march(w.nt)
            snaps[prec] = (sv.snapshots().astype(np.complex128), sv.read(F.READ_NORMS))
            sv.close()
        a, b = snaps[F.F32_COMP][0], snaps[F.F64][0]
        errs.append(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)))
        n64 = snaps[F.F64][1]
        nerrs.append(float(np.max(np.abs(norms - n64)) / max(np.max(np.abs(n64)), 1e-300)))
    f64 = None
    if args.compare_f64:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for w in ws_list:
            s64 = F.Solver(F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0,
                                    k=w.k, init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center,
                                    tstep=-1))
            s64.set_boundary()
            s64.march(w.nt)
            s64.read(F.READ_NORMS)
            s64.close()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        f64 = {"value": updates / dt, "unit": UNIT, "how": "same instances, one FP64 plan each, back to back "
                                                           "(wall clock, plan + boundary + march + norms)"}
    F.fdtd_destroy(plan)
    del buf
    ach = 16 * updates / (t_march * 1e-3) / 1e9
    out = {"metric": METRIC, "value": updates * steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
           "steps": steps, "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c64-compensated (FP64 boundary and norms)",
           "data": "synthetic",
           "config": {"workload": name, "instances": len(ws_list), "updates_per_step": updates,
                      "march": "CUDA graph of the persistent launches (fdtd_march_graph)",
                      "autotune": tuned,
                      "l2": f"inputs larger than L2 (plan workspace {nbytes.value / 1e9:.1f} GB)"},
           "roofline": {"kernel": "k_march_f32c", "bound": "hbm", "achieved": ach, "peak": peaks.get("hbm_gbs"),
                        "unit": "GB/s", "frac": ach / peaks.get("hbm_gbs", 6800.0), "traffic": None,
                        "bytes_per_update": 16, "launch_ms": t_march, "peak_source": src},
           "boundary_ms": t_bnd, "march_ms": t_march, "march_only_value": updates / (t_march * 1e-3),
           "error_vs_fp64": {"instances": pick, "stored_rows_rel_l2_max": max(errs), "norms_rel_max": max(nerrs),
                             "per_instance": [{"i": i, "nx": ws_list[i].nx, "nt": ws_list[i].nt, "D": ws_list[i].D,
                                               "rel_l2": e, "norms_rel": ne}
                                              for i, e, ne in zip(pick, errs, nerrs)],
                             "how": "~512 stored rows of each instance (the 3 largest by updates and the "
                                    "smallest) marched alone in complex64 and FP64; norms of the timed plan "
                                    "vs FP64"},
           "clocks": clocks}
    if f64:
        out["fp64_same_instances"] = f64
    return out


def surrogate_variant(args, steps, warmup, peaks, src):
    """Training and inference throughput of one surrogate network (4 -> 512 x 4
    GELU -> 8704, BF16 tensor cores) on random inputs of the surrogate's shape."""
    import torch

    from paper_1707_05943_gb300 import fdtd as F, surrogate as S
    batch = 512
    net = S.Net(S.DIMS, seed=1)
    x = torch.rand(batch, 4, device="cuda") * 2 - 1
    t = torch.randn(batch, S.N_OUT, device="cuda")
    y = torch.empty(batch, S.N_OUT, device="cuda")
    st = torch.cuda.ExternalStream(net.sp)
    for _ in range(warmup * 10):
        net.train_step(x, t, 1e-4)
    torch.cuda.synchronize()
    n_steps = 200 * steps
    sampler = ClockSampler(0)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    sampler.start()
    e0.record(st)
    for _ in range(n_steps):
        net.train_step(x, t, 1e-4)
    e1.record(st)
    for _ in range(n_steps):
        net.forward(x, y)
    e2.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    F.fdtd_mlp_status(net.sp)
    ms_train = e0.elapsed_time(e1) / n_steps
    ms_inf = e1.elapsed_time(e2) / n_steps
    fl = 2 * batch * sum(S.DIMS[i] * S.DIMS[i + 1] for i in range(1, len(S.DIMS) - 1))
    ach = 3 * fl / (ms_train * 1e-3) / 1e12
    out = {"metric": "surrogate training samples/s (BF16 tensor cores)", "value": batch / (ms_train * 1e-3),
           "unit": "samples/s", "n_gpus": 1, "steps": n_steps, "warmup": warmup * 10,
           "ms_per_step": ms_train, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16 (FP32 accumulation, FP32 master weights)", "data": "synthetic",
           "config": {"workload": "surrogate_4x512x4_8704", "batch": batch,
                      "l2": "weights and activations L2-resident (training step; no flush)"},
           "inference": {"value": batch / (ms_inf * 1e-3), "unit": "samples/s", "ms_per_batch": ms_inf},
           "roofline": {"kernel": "k_gemm_nt_tma (all GEMMs of the step)", "bound": "tensor", "achieved": ach,
                        "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                        "frac": ach / peaks.get("bf16_tflops", 1900.0), "traffic": None, "peak_source": src},
           "clocks": clocks}
    del net
    return out


def f64_variant(args, rows, alu_fp64):
    """The native FP64 march (FDTD_F64, k_march_f64) on `rows` - 1 rows from the middle
    of the large workload (rows 1 .. nt/2, untimed, come first: a row's cost grows with n,
    since the source terms act only inside the light cone j < n + D, so the middle rows
    cost the average of the full march), in the default launch size, with CUDA events
    around every timed launch on the plan's stream."""
    import torch

    from paper_1707_05943_gb300 import fdtd as F
    rpl = args.rows_per_launch
    pre = (W.LARGE.nt // 2) // rpl * rpl
    w = W.LARGE.with_(nt=rows + pre)
    stream = torch.cuda.Stream()
    cfg = F.Config(nx=w.nx, nt=w.nt, D=w.D, delta=w.delta, gamma=w.gamma, omega0=w.omega0, k=w.k,
                   init_cond=w.init_cond, alpha=w.alpha, sigma=w.sigma, center=w.center, tstep=-1,
                   rows_per_launch=rpl, precision=F.F64)
    s = F.Solver(cfg, stream=stream)
    ev = []

    s.set_boundary()
    s.march(pre)  # untimed: takes the march to the middle rows and warms the GPU up
    stream.synchronize()
    sampler = ClockSampler(env_rank()[2])
    sampler.start()
    done = 1 + pre
    while done < w.nt:
        n = min(rpl, w.nt - done)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.march(n)
        b.record(stream)
        ev.append((a, b, n))
        done += n
    stream.synchronize()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    upd = w.nx * sum(n for _, _, n in ev)
    full = [a.elapsed_time(b) for a, b, n in ev if n == rpl] or [ms]
    launch_ms = sum(full) / len(full)
    cnt = march_work(w, pre + 1, w.nt)
    ins, fl = work_of(cnt, F64_INSTR), work_of(cnt, F64_FLOPS)
    ach = ins / (ms * 1e-3) / 1e12
    s.close()
    del s
    return {"value": upd / (ms * 1e-3), "unit": UNIT, "dtype": "f64", "kernel": "k_march_f64",
            "rows_measured": rows - 1, "rows_from": pre + 1, "march_ms": ms, "launch_ms": launch_ms,
            "roofline": {"bound": "alu", "achieved": ach, "peak": alu_fp64 / 2,
                         "unit": "T FP64-pipe instructions/s (DADD, DMUL, DFMA each 1)",
                         "frac": ach / (alu_fp64 / 2), "fp64_instr_per_update": ins / cnt["updates"],
                         "flops_per_update": fl / cnt["updates"],
                         "flops_frac": fl / (ms * 1e-3) / 1e12 / alu_fp64,
                         "peak_source": "measured in this run (fdtd_alu_probe, FP64 FMA) / 2 flops per FMA"},
            "how": f"march only, rows {pre + 1}..{w.nt - 1} of {W.LARGE.name} (rows 1..{pre} marched untimed first), "
                   "CUDA events per launch", "clocks": clocks}


def solver_grid(s) -> int:
    # column split entries copied host->device by fdtd_set_boundary (grid+1 int64)
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


if __name__ == "__main__":
    main()

"""Throughput of the coupled three-lattice step (MLUPS) on GB300.

Default workload: the 2048x1024 drop-in-shear grid (R = 192, W = 5, Ca = 0.1,
beta = 0.3, Gamma0 = 0.3, Re = 0.1, Pe_s = 10), FP32 populations, coupled
f + h + g lattices with moving walls.  One bench step = one LBM time step of
the whole grid (one fused kernel launch).  The population buffers (453 MB)
exceed L2, so no explicit flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--workload sphere3d (sphere3d-384) times the D3Q27 phase-field + surfactant
step on a 256^3 (384^3) advected spherical drop instead.

--impl reference times the FP64 CPU oracle on the host cores instead (each
step a bounded window of the same workload).  Under torchrun (N > 1) every
rank runs an independent replica (the single-grid path has no exchange step);
value = total cell updates of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes per coupled cell update: 27 populations read and written
# once (the 16-bit format also moves two 32-bit zeroth moments per cell,
# 120 B in all, which count as traffic above the algorithmic figure)
BYTES_PER_CELL = {"f32": 216, "f16s": 108, "bf16s": 108}
METRIC = "coupled MLUPS"
UNIT = "MLUPS"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest value of x over all ranks (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells_per_rank, steps, seconds):
    """Cell updates of all ranks per second of the slowest rank, in millions."""
    return world * cells_per_rank * steps / seconds / 1e6


def make_case(name):
    from paper_2504_09024_gb300 import workloads as W
    if name == "2048x1024":
        return W.shear_drop_2048x1024(Ca=0.1)
    if name == "512x256":
        return W.shear_drop_512x256()
    raise SystemExit(f"unknown workload {name}")


def traffic_record(kernel_name):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (hash match); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel_name)
    except Exception:
        return None
    if not rec:
        return None
    from paper_2504_09024_gb300 import build as B
    if rec.get("source_hash") != B.source_hash("3d" if kernel_name.startswith("k3_") else "2d"):
        return None
    return rec


def cpu_baseline(case, budget_s=15.0):
    """FP64 oracle on the host cores over a bounded window of the workload."""
    import oracle
    from paper_2504_09024_gb300 import workloads as W
    nx, ny = case.phys.nx, case.phys.ny
    # window: full height band through the drop centre, width chosen by a probe
    def window(wx, wy):
        x0 = int(max(0, nx // 2 - int(case.meta.get("R", 0)) - wx // 2))
        x0 = min(x0, nx - wx)
        y0 = (ny - wy) // 2
        sl = (slice(y0, y0 + wy), slice(x0, x0 + wx))
        phys = W.Physics(**{**case.phys.as_dict(), "nx": wx, "ny": wy})
        return phys, [a[sl].copy() for a in (case.phi, case.c, case.ux, case.uy)]

    phys, arrs = window(min(nx, 256), min(ny, 128))
    s = oracle.Sim(phys)
    s.init(*arrs)
    s.step(1)
    t0 = time.perf_counter()
    s.step(2)
    per_cell_step = (time.perf_counter() - t0) / (2 * phys.nx * phys.ny)
    s.close()
    steps = max(1, int(budget_s / (per_cell_step * phys.nx * phys.ny)))
    s = oracle.Sim(phys)
    s.init(*arrs)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    s.close()
    mlups = phys.nx * phys.ny * steps / dt / 1e6
    return {"value": mlups, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} steps of a {phys.nx}x{phys.ny} window of the {nx}x{ny} "
                      f"workload through the drop interface ({dt:.1f} s)"}


def run_reference_3d(args, world):
    """The 3-D oracle on the host cores: the sphere workload scaled down to a
    box whose (warm-up + timed) steps fit the budget."""
    import oracle
    n_full = SPHERE3D_N[args.workload]
    probe = sphere3d_case(16)
    s = oracle.Sim3(16, 16, 16, W=probe.W, M_phi=probe.M_phi, D_s=probe.D_s)
    s.init(probe.phi, probe.c, *probe.u)
    s.step(1)
    t0 = time.perf_counter()
    s.step(3)
    t_cell = (time.perf_counter() - t0) / (3 * 16 ** 3)
    s.close()
    total_steps = args.steps + args.warmup
    n = int((args.ref_budget / (total_steps * t_cell)) ** (1.0 / 3.0))
    n = max(8, min(n_full, n - n % 4))
    case = sphere3d_case(n)
    s = oracle.Sim3(n, n, n, W=case.W, M_phi=case.M_phi, D_s=case.D_s)
    s.init(case.phi, case.c, *case.u)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    s.close()
    value = n ** 3 * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": "D3Q27 phase-field + surfactant MLUPS", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"sphere_{n_full}^3_l1",
                   "grid": f"{n_full}x{n_full}x{n_full}", "sample": f"the same drop scaled to {n}^3",
                   "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: one oracle step of the workload scaled to {n}^3"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    if args.workload in SPHERE3D_N:
        return run_reference_3d(args, world)
    case = make_case(args.workload)
    from paper_2504_09024_gb300 import workloads as W
    nx, ny = case.phys.nx, case.phys.ny
    total_steps = args.steps + args.warmup
    # size the per-step window so the whole run takes about args.ref_budget seconds
    probe = W.Physics(**{**case.phys.as_dict(), "nx": 128, "ny": 64})
    s = oracle.Sim(probe)
    s.init(*(a[(ny - 64) // 2:(ny + 64) // 2, :128].copy() for a in (case.phi, case.c, case.ux, case.uy)))
    s.step(1)
    t0 = time.perf_counter()
    s.step(3)
    t_cell = (time.perf_counter() - t0) / (3 * 128 * 64)
    s.close()
    cells = max(64, min(nx * ny, int(args.ref_budget / (total_steps * t_cell))))
    wy = max(4, min(ny, int(math.sqrt(cells / 2))))
    wx = max(4, min(nx, cells // wy))
    y0, x0 = (ny - wy) // 2, max(0, (nx - wx) // 2)
    sl = (slice(y0, y0 + wy), slice(x0, x0 + wx))
    phys = W.Physics(**{**case.phys.as_dict(), "nx": wx, "ny": wy})
    s = oracle.Sim(phys)
    s.init(*(a[sl].copy() for a in (case.phi, case.c, case.ux, case.uy)))
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    s.close()
    value = wx * wy * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": case.name, "grid": f"{nx}x{ny}",
                   "sample": f"{wx}x{wy} window per step", "parallelism": "host threads"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"each step: one oracle step of a {wx}x{wy} window of the "
                                   f"{nx}x{ny} workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ensemble(args, rank, world, local_rank):
    """One ensemble of drop-in-shear runs (uneven grids) sharded over the
    ranks: every run is stepped by exactly one rank (runs dealt out by cell
    count), each rank's runs as one batch in the form and launch shape
    lbm_batch_autotune picks, and the per-run diagnostics gathered to rank 0
    at the end.  value = cell updates of all runs per second of the slowest
    rank; runs_per_hour converts the step time to runs of RUN_STEPS steps."""
    import torch
    from paper_2504_09024_gb300 import ensemble, lbm, workloads as W

    RUN_STEPS = 20000
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    nruns = int(args.workload[len("ensemble"):] or 64)
    draws = W.ensemble_draws(nruns=nruns, seed=W.CASE_SEED)
    all_cases = [W.ensemble_case(d, steps=RUN_STEPS) for d in draws]
    ncell_all = sum(c.phys.nx * c.phys.ny for c in all_cases)
    owned = ensemble.shard([c.phys.nx * c.phys.ny for c in all_cases], world)[rank]
    cases = [all_cases[r] for r in owned]
    ncell = sum(c.phys.nx * c.phys.ny for c in cases)
    stream = torch.cuda.Stream()
    b = lbm.Batch([c.phys for c in cases], stream=stream.cuda_stream)
    for r, c in zip(b.runs, cases):
        r.init(c.phi, c.c, c.ux, c.uy)
    if args.tile_x or args.seg_y:
        if args.batch_form:
            b.set_form(lbm.LBM_BATCH_CHAINS if args.batch_form == "chains"
                       else lbm.LBM_BATCH_PERSISTENT)
        b.set_launch_shape(args.tile_x, args.seg_y)
        tuned = None
    else:
        tx, sy, tms = b.autotune(steps=8)
        tuned = {"tile_x": tx, "seg_y": sy, "ms_per_step": tms}
    bx, seg, blocks, tiles = b.launch_shape()
    b.step(args.warmup)
    b.sync()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms_max = max_over_ranks(e0.elapsed_time(e1), dist)
    ms_step = ms_max / args.steps
    value = ncell_all * args.steps / (ms_max * 1e-3) / 1e6

    # end to end through the public API: every run initialised from pinned
    # host fields, K batched steps, every run's fields read back + diagnostics
    host_in = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (c.phi, c.c, c.ux, c.uy)] for c in cases]
    host_out = [[torch.empty((c.phys.ny, c.phys.nx), dtype=torch.float64).pin_memory()
                 for _ in range(5)] for c in cases]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, hin in zip(b.runs, host_in):
        lbm.lbm_init_fields(r.ctx, *hin)
    b.step(args.steps)
    diags = []
    for r, hout in zip(b.runs, host_out):
        lbm.lbm_get_fields(r.ctx, *hout)
        diags.append(r.diagnostics())
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    # host bytes of the whole job (each rank copies its own runs)
    h2d = sum(c.phys.nx * c.phys.ny * 8 * 4 for c in all_cases)
    d2h = sum(c.phys.nx * c.phys.ny * 8 * 5 for c in all_cases) + 128 * nruns
    gathered = ensemble.gather_rows(
        {r: [d["sum_phi"], d["sum_c"], d["D"], d["nonfinite"]] for r, d in zip(owned, diags)},
        dist)

    peak, peak_kind = peaks()
    bpc = BYTES_PER_CELL[args.dtype]
    achieved = bpc * ncell / (ms_step * 1e-3) / 1e9
    # kernels a rank launches per step: one per run in the chains form (and
    # one counter update per graph), one per table of 64 runs in the
    # persistent form
    form = b.form
    per_step = len(cases) if form == lbm.LBM_BATCH_CHAINS else (len(cases) + 63) // 64
    launches = args.steps * per_step + (args.steps + 31) // 32
    grids = {}
    for c in all_cases:
        k = f"{c.phys.nx}x{c.phys.ny}"
        grids[k] = grids.get(k, 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": f"ensemble of {nruns} drop-in-shear runs", "runs": nruns,
                   "grids": grids, "cells_per_step": ncell_all,
                   "kernel": ("k_sweep2 per run (chains of single-run launches in graphs)"
                              if form == lbm.LBM_BATCH_CHAINS else
                              "k_sweep2_batch (one persistent launch per step in graphs)"),
                   "form": "chains" if form == lbm.LBM_BATCH_CHAINS else "persistent",
                   "launch_shape": [bx, seg], "persistent_blocks": blocks, "tiles": tiles,
                   "launch_shape_from": "lbm_batch_autotune" if tuned else "command line",
                   "l2": "populations exceed the 129 MB L2; no flush",
                   "parallelism": (f"one ensemble sharded over {world} ranks by cell count, "
                                   "diagnostics gathered" if world > 1 else "single GPU")},
        "runs_per_hour": nruns * 3600.0 / (RUN_STEPS * ms_step * 1e-3),
        "run_steps": RUN_STEPS,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "bytes_per_cell": bpc, "traffic": None},
        "e2e": {"value": whole_job_mlups(world, ncell, args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "lbm_init_fields of every run from pinned host fields + "
                        "lbm_batch_step(K) + lbm_get_fields and lbm_diagnostics of every run"},
        "gpu_launches": launches,
        "clocks": clk,
        "check": ({"runs_reported": len(gathered),
                   "nonfinite": int(sum(v[3] for v in gathered.values()))}
                  if gathered is not None else None),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(all_cases[0], args.cpu_budget)
    b.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def timed_regions(step_fn, stream, k, repeats, dist=None):
    """Times `repeats` regions of exactly k steps with CUDA events on the
    launching stream, each bracketed by a barrier and device synchronisation;
    returns the per-region times (ms, max over ranks)."""
    import torch
    out = []
    for _ in range(repeats):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_fn(k)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        out.append(max_over_ranks(e0.elapsed_time(e1), dist))
    return out


def bench_single(case, dtype, args, stream, dist=None, autotune=True):
    """One context on the workload: autotuned launch shape, W warm-up steps
    plus one untimed pass of K steps (it captures the step graphs the timed
    regions replay), then `repeats` timed regions of K steps.  Returns the
    context and the per-region times (ms)."""
    from paper_2504_09024_gb300 import lbm
    dtype_code = {"f32": lbm.LBM_F32, "f16s": lbm.LBM_F16S, "bf16s": lbm.LBM_BF16S}[dtype]
    kern = {"auto": lbm.LBM_KERNEL_AUTO, "tma": lbm.LBM_KERNEL_TMA, "fused": lbm.LBM_KERNEL_FUSED,
            "split": lbm.LBM_KERNEL_SPLIT}[args.kernel]
    sim = lbm.Sim(case.phys, dtype=dtype_code, kernel=kern, stream=stream.cuda_stream)
    if args.tile_x or args.seg_y:
        sim.set_launch_shape(args.tile_x, args.seg_y)
    sim.init(case.phi, case.c, case.ux, case.uy)
    tuned = None
    if autotune and not (args.tile_x or args.seg_y) and sim.kernel != lbm.LBM_KERNEL_SPLIT:
        # the library's autotuner picks the launch shape on the live state
        # (and puts the state back) before the warm-up
        tx, sy, tms = sim.autotune(steps=32)
        tuned = {"tile_x": tx, "seg_y": sy, "ms_per_step": tms}
    sim.step(args.warmup)
    sim.step(args.steps)
    sim.sync()
    times = timed_regions(sim.step, stream, args.steps, args.repeats, dist)
    return sim, times, tuned


def kernel_name(sim, dtype):
    from paper_2504_09024_gb300 import lbm
    if dtype != "f32":
        return "k_sweep2_16"
    return {lbm.LBM_KERNEL_TMA: "k_sweep2", lbm.LBM_KERNEL_FUSED: "k_fused_sweep",
            lbm.LBM_KERNEL_SPLIT: "k_collide"}[sim.kernel]


def roofline(dtype, ncell, ms_step, kname):
    peak, peak_kind = peaks()
    bpc = BYTES_PER_CELL[dtype]
    achieved = bpc * ncell / (ms_step * 1e-3) / 1e9
    tr = traffic_record(kname)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs", "bytes_per_cell": bpc,
            "traffic": tr["bytes_per_launch"] if tr else None}


def ensemble_comparison(args, stream):
    """The 64-run ensemble (uneven grids) in one batch against the same runs
    stepped one context at a time; FP32, launch shapes from the autotuners.
    Returns runs/hour of each form at RUN_STEPS steps per run."""
    import torch
    from paper_2504_09024_gb300 import lbm, workloads as W
    RUN_STEPS = 20000
    draws = W.ensemble_draws(nruns=64, seed=W.CASE_SEED)
    cases = [W.ensemble_case(d, steps=RUN_STEPS) for d in draws]
    ncell = sum(c.phys.nx * c.phys.ny for c in cases)
    k = 64
    b = lbm.Batch([c.phys for c in cases], stream=stream.cuda_stream)
    for r, c in zip(b.runs, cases):
        r.init(c.phi, c.c, c.ux, c.uy)
    b.autotune(steps=8)
    b.step(k)
    b.sync()
    t_batch = statistics.median(timed_regions(b.step, stream, k, 3)) / k
    b.close()
    # one context at a time: every run's grid on its own (runs of equal grid
    # size cost the same; each size is timed once on one of its runs)
    by_grid = {}
    for c in cases:
        by_grid.setdefault((c.phys.nx, c.phys.ny), []).append(c)
    t_seq = 0.0
    for (nx, ny), cs in by_grid.items():
        sim = lbm.Sim(cs[0].phys, stream=stream.cuda_stream)
        sim.init(cs[0].phi, cs[0].c, cs[0].ux, cs[0].uy)
        sim.autotune(steps=32)
        sim.step(k)
        sim.sync()
        t_one = statistics.median(timed_regions(sim.step, stream, k, 3)) / k
        t_seq += t_one * len(cs)
        sim.close()
    torch.cuda.synchronize()
    return {"runs": len(cases), "cells_per_step": ncell, "run_steps": RUN_STEPS,
            "batched": {"mlups": ncell / (t_batch * 1e-3) / 1e6,
                        "runs_per_hour": len(cases) * 3600.0 / (RUN_STEPS * t_batch * 1e-3)},
            "one_context_at_a_time": {
                "mlups": ncell / (t_seq * 1e-3) / 1e6,
                "runs_per_hour": len(cases) * 3600.0 / (RUN_STEPS * t_seq * 1e-3)},
            "timing": f"median of 3 regions of {k} steps, CUDA events"}


# The D3Q27 phase-field + surfactant step (include/lbm3.h): 27 fixed-point
# words per lattice read and written once per cell update, two lattices.
BYTES_PER_CELL_3D = 432
SPHERE3D_N = {"sphere3d": 256, "sphere3d-384": 384,
              "sphere3d-128": 128}  # 128^3 (0.9 GB, above L2): the profiler's small case


def sphere3d_case(n):
    """Spherical drop R = n/4 in an n^3 periodic box with an l = 1 surface
    mode of surfactant, advected by a uniform velocity (the 3-D form of the
    advected drop of Sec. 4.1)."""
    from paper_2504_09024_gb300 import workloads as W
    return W.sphere_surface_mode(n=n, W=4.0, D_s=0.1, M_phi=0.05, mode=1, u=(0.02, -0.013, 0.009))


def cpu_baseline_3d(budget_s=15.0):
    """The 3-D FP64 oracle on the host cores: the same workload scaled down to
    a 32^3 box (R = 8), as many steps as fit the budget."""
    import oracle
    case = sphere3d_case(32)
    s = oracle.Sim3(32, 32, 32, W=case.W, M_phi=case.M_phi, D_s=case.D_s)
    s.init(case.phi, case.c, *case.u)
    t0 = time.perf_counter()
    s.step(2)
    per_step = (time.perf_counter() - t0) / 2
    steps = max(1, int(budget_s / per_step))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    s.close()
    return {"value": 32 ** 3 * steps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{steps} steps of the same workload scaled to a 32^3 box "
                                        f"(R = 8), {dt:.1f} s"}


def bench_sphere3d(n, args, stream, dist=None):
    """Autotuned 3-D context on the n^3 sphere: W warm-up steps and one untimed
    pass of K, then `repeats` timed regions of K steps (CUDA events on the
    library's stream), and the end-to-end leg through the public API."""
    import torch
    from paper_2504_09024_gb300 import lbm3
    case = sphere3d_case(n)
    g = lbm3.Sim3(n, n, n, W=case.W, M_phi=case.M_phi, D_s=case.D_s, u=case.u,
                  stream=stream.cuda_stream)
    if args.rows or args.seg_z:
        lbm3.lbm3_set_launch_shape(g.ctx, args.rows, args.seg_z)
        rows, seg = lbm3.lbm3_get_launch_shape(g.ctx)
    else:
        rows, seg, tms = lbm3.lbm3_autotune(g.ctx, 8)
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (case.phi, case.c)]
    lbm3.lbm3_init_fields(g.ctx, *[a.numpy() for a in host_in])
    g.step(args.warmup)
    g.step(args.steps)
    g.synchronize()
    times = timed_regions(g.step, stream, args.steps, args.repeats, dist)
    ms_step = statistics.median(times) / args.steps
    host_out = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm3.lbm3_init_fields(g.ctx, *[a.numpy() for a in host_in])
    g.step(args.steps)
    lbm3.lbm3_get_fields(g.ctx, *[a.numpy() for a in host_out])
    sums = g.sums()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    peak, peak_kind = peaks()
    achieved = BYTES_PER_CELL_3D * n ** 3 / (ms_step * 1e-3) / 1e9
    tr = traffic_record("k3_step")
    out = {
        "case": case, "ms_step": ms_step, "times": times, "e2e_s": e2e_s,
        "h2d": sum(a.numel() * 8 for a in host_in), "d2h": sum(a.numel() * 8 for a in host_out) + 24,
        "launch_shape": [rows, seg], "sums": sums,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "bytes_per_cell": BYTES_PER_CELL_3D,
                     "traffic": tr["bytes_per_launch"] if tr else None},
    }
    g.close()
    return out


def run_sphere3d(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    n = SPHERE3D_N[args.workload]
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    r = bench_sphere3d(n, args, stream, dist)
    clk = clocks.stop()
    ncell = n ** 3
    line = {
        "metric": "D3Q27 phase-field + surfactant MLUPS", "value": whole_job_mlups(world, ncell, args.steps, r["ms_step"] * args.steps * 1e-3),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fixed-point int32 storage, f32 arithmetic", "data": "synthetic",
        "config": {"workload": r["case"].name, "grid": f"{n}x{n}x{n}", "cells": ncell,
                   "lattices": "f+h (D3Q27) under a uniform prescribed velocity",
                   "kernel": "k3_step", "launch_shape": r["launch_shape"],
                   "launch_shape_from": "command line" if (args.rows or args.seg_z) else "lbm3_autotune",
                   "timed_regions": f"median of {args.repeats} regions of {args.steps} steps",
                   "l2": f"populations (2 x {ncell * 216 / 1e9:.1f} GB) exceed the 129 MB L2; no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": r["roofline"],
        "e2e": {"value": whole_job_mlups(world, ncell, args.steps, r["e2e_s"]), "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"] / args.steps, "d2h_bytes_per_step": r["d2h"] / args.steps,
                "what": "lbm3_init_fields from pinned host fields + lbm3_step(K) + lbm3_get_fields "
                        "to pinned host + lbm3_sums"},
        "gpu_launches": args.steps,
        "clocks": clk,
        "check": {"sum_phi": r["sums"]["sum_phi"], "sum_c": r["sums"]["sum_c"],
                  "invalid": r["sums"]["nonfinite"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_3d(args.cpu_budget)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2504_09024_gb300 import lbm

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()

    case = make_case(args.workload)
    nx, ny = case.phys.nx, case.phys.ny
    ncell = nx * ny
    stream = torch.cuda.Stream()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    sim, times, tuned = bench_single(case, args.dtype, args, stream, dist)
    clk = clocks.stop()
    ms_region = statistics.median(times)
    value = whole_job_mlups(world, ncell, args.steps, ms_region * 1e-3)
    ms_step = ms_region / args.steps
    launches = lbm.lbm_launches_per_step(sim.ctx)

    # end-to-end through the public API with pinned host buffers: initialise
    # from host fields, run the same number of steps, read fields + diagnostics
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (case.phi, case.c, case.ux, case.uy)]
    host_out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(5)]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_init_fields(sim.ctx, *host_in)
    sim.step(args.steps)
    lbm.lbm_get_fields(sim.ctx, *host_out)
    diag = sim.diagnostics()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    h2d = sum(a.numel() * 8 for a in host_in)
    d2h = sum(a.numel() * 8 for a in host_out) + 128

    kname = kernel_name(sim, args.dtype)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": case.name, "grid": f"{nx}x{ny}", "cells": ncell,
                   "lattices": "f+h+g coupled", "kernel": kname,
                   "launch_shape": list(lbm.lbm_get_launch_shape(sim.ctx)),
                   "launch_shape_from": "lbm_autotune" if tuned else "command line",
                   "timed_regions": f"median of {args.repeats} regions of {args.steps} steps "
                                    f"({', '.join(f'{t / args.steps * 1e3:.2f}' for t in times)} "
                                    f"us/step); W warm-up steps and one untimed {args.steps}-step "
                                    f"pass before them",
                   "l2": "populations (2 x 226 MB) exceed the 129 MB L2; no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline(args.dtype, ncell, ms_step, kname),
        "e2e": {"value": whole_job_mlups(world, ncell, args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                "what": "lbm_init_fields from pinned host fields + lbm_step(K) + lbm_get_fields "
                        "to pinned host + lbm_diagnostics"},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "check": {"sum_phi": diag["sum_phi"], "nonfinite": diag["nonfinite"]},
    }
    sim.close()
    if rank == 0 and world == 1 and args.dtype == "f32" and not args.no_extras:
        # the same workload with 16-bit storage, and the batched ensemble
        # against one context at a time (extra keys of the same line)
        for dt in ("f16s", "bf16s"):
            s16, t16, _ = bench_single(case, dt, args, stream)
            ms16 = statistics.median(t16) / args.steps
            line[dt] = {"value": ncell / (ms16 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms16,
                        "launch_shape": list(lbm.lbm_get_launch_shape(s16.ctx)),
                        "vs_f32": ms_step / ms16,
                        "roofline": roofline(dt, ncell, ms16, "k_sweep2_16")}
            s16.close()
        line["ensemble64"] = ensemble_comparison(args, stream)
        r3 = bench_sphere3d(256, args, stream)
        line["sphere3d"] = {"workload": r3["case"].name, "value": 256 ** 3 / (r3["ms_step"] * 1e-3) / 1e6,
                            "unit": UNIT, "ms_per_step": r3["ms_step"],
                            "launch_shape": r3["launch_shape"], "roofline": r3["roofline"],
                            "what": "D3Q27 phase-field + surfactant lattices, fixed-point storage, "
                                    "uniform prescribed velocity (k3_step, one launch per step)"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case, args.cpu_budget)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="2048x1024")
    ap.add_argument("--dtype", choices=["f32", "f16s", "bf16s"], default="f32")
    ap.add_argument("--kernel", choices=["auto", "tma", "fused", "split"], default="auto")
    ap.add_argument("--tile-x", type=int, default=0)
    ap.add_argument("--seg-y", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0, help="3-D workloads: tile rows (6, 10, 18)")
    ap.add_argument("--seg-z", type=int, default=0, help="3-D workloads: planes per block")
    ap.add_argument("--batch-form", choices=["chains", "persistent"], default=None,
                    help="ensemble with a given launch shape: the batched form (default persistent)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=90.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the 16-bit and ensemble keys of the default line")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of K steps; the median is reported")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload.startswith("ensemble"):
        return run_ensemble(args, rank, world, local_rank)
    if args.workload in SPHERE3D_N:
        return run_sphere3d(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())

"""Per-run metrics log: one JSON object per line (JSONL).

A record holds the run's parameters (once, in its first record), the step,
the FP64 reductions of the library's diagnostics (sum phi, sum c, the
deformation D and the axes L and B), the throughput since the previous
record (MLUPS, and GB/s from the populations each cell update reads and
writes), the storage type and the launch shape.  The statistics come from
lbm_diagnostics (device reductions); this module only times and formats.

    log = MetricsLog("PROGRESS.jsonl", sim, run="drop-7")
    for _ in range(10):
        sim.step(1000)
        log.record()
"""
from __future__ import annotations

import json
import time

from . import lbm, workloads as W

# Algorithmic population bytes of one cell update: every population read
# once and written once, 9 per lattice, 4 bytes in FP32 storage and 2 in the
# 16-bit formats (the figure the roofline of the step is quoted against).
def bytes_per_cell(dtype: int, coupled: bool) -> int:
    lattices = 3 if coupled else 2
    return 2 * 9 * lattices * (4 if dtype == lbm.LBM_F32 else 2)


class MetricsLog:
    def __init__(self, path: str, sim: "lbm.Sim", run: str = "", extra: dict | None = None):
        self.path = path
        self.sim = sim
        self.run = run
        self.extra = dict(extra or {})
        self._t = None
        self._step = None
        self._first = True

    def _params(self) -> dict:
        p = self.sim.params
        return {name: getattr(p, name) for name, _ in p._fields_}

    def record(self, **fields) -> dict:
        """Synchronise the run, take its diagnostics and append one line."""
        self.sim.sync()
        now = time.perf_counter()
        step = int(self.sim.t)
        d = self.sim.diagnostics()
        coupled = self.sim.mode != lbm.LBM_FIXED_U
        dtype = int(self.sim.params.dtype)
        rec = {"run": self.run, "step": step, "sum_phi": d["sum_phi"], "sum_c": d["sum_c"],
               "D": d["D"], "L": d["L"], "B": d["B"], "nonfinite": d["nonfinite"],
               "dtype": {lbm.LBM_F32: "f32", lbm.LBM_F16S: "f16s",
                         lbm.LBM_BF16S: "bf16s"}.get(dtype, str(dtype)),
               "launch_shape": list(lbm.lbm_get_launch_shape(self.sim.ctx)),
               "cells_per_thread": self.sim.cells_per_thread,
               "store_mode": self.sim.store_mode}
        if self._t is not None and step > self._step:
            dt = now - self._t
            cells = self.sim.nx * self.sim.ny * (step - self._step)
            rec["MLUPS"] = cells / dt / 1e6
            rec["GBps"] = cells * bytes_per_cell(dtype, coupled) / dt / 1e9
        if self._first:
            rec["params"] = self._params()
            rec.update(self.extra)
            self._first = False
        rec.update(fields)
        with open(self.path, "a") as f:
            f.write(json.dumps(rec, default=float) + "\n")
        # time the next interval from after the diagnostics
        self._t = time.perf_counter()
        self._step = step
        return rec


WORKLOADS = {
    "shear512": lambda steps: W.shear_drop_512x256(steps),
    "shear2048": lambda steps: W.shear_drop_2048x1024(Ca=0.1, steps=steps),
}


def main(argv=None):
    """Run a named workload and log a record every `every` steps, e.g. the
    512 x 256 drop's deformation D(t) over 40,000 FP32 steps:

        python -m paper_2504_09024_gb300.metrics --workload shear512 \\
            --steps 40000 --every 2000 --out PROGRESS.jsonl
    """
    import argparse
    ap = argparse.ArgumentParser(description="JSONL metrics of one run")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="shear512")
    ap.add_argument("--steps", type=int, default=40000)
    ap.add_argument("--every", type=int, default=2000)
    ap.add_argument("--dtype", choices=["f32", "f16s", "bf16s"], default="f32")
    ap.add_argument("--out", default="PROGRESS.jsonl")
    args = ap.parse_args(argv)
    dt = {"f32": lbm.LBM_F32, "f16s": lbm.LBM_F16S, "bf16s": lbm.LBM_BF16S}[args.dtype]
    case = WORKLOADS[args.workload](args.steps)
    sim = lbm.Sim(case.phys, dtype=dt)
    sim.init(case.phi, case.c, case.ux, case.uy)
    log = MetricsLog(args.out, sim, run=case.name, extra={"meta": case.meta})
    gamma_dot = case.meta.get("gamma_dot")
    rec = log.record(t_star=0.0)
    print(json.dumps({k: rec[k] for k in ("step", "D", "sum_phi", "sum_c")}))
    done = 0
    while done < args.steps:
        n = min(args.every, args.steps - done)
        sim.step(n)
        done += n
        rec = log.record(t_star=done * gamma_dot if gamma_dot else None)
        print(json.dumps({k: rec[k] for k in ("step", "D", "sum_phi", "sum_c", "MLUPS")}))
    sim.close()
    return 0


if __name__ == "__main__":
    main()

"""FP64 oracle reference of the 2048x1024 precision workload, computed in a
background process while the rest of the GPU suite runs.

The FP64 oracle needs about 10-15 minutes on the host cores for 5000 steps of
the 2048 x 1024 drop, so the suite starts it as soon as collection finishes
(tests/conftest.py) and the precision test collects the result at the end.
Run as a script, it computes one reference and writes it to an .npz file:

    python tests/long_reference.py OUT.npz CA STEPS
"""
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

_jobs = {}


def _out_path(Ca, steps):
    d = os.environ.get("LBM_REFERENCE_DIR") or os.path.join(tempfile.gettempdir(),
                                                             f"lbm_ref_{os.getpid()}")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"shear_2048x1024_Ca{Ca:g}_{steps}.npz")


def start(Ca, steps):
    """Start the background oracle run (once per Ca, steps).  A finished
    reference already in LBM_REFERENCE_DIR (written by this script) is
    reused."""
    key = (Ca, steps)
    if key in _jobs:
        return _jobs[key]
    out = _out_path(Ca, steps)
    if os.environ.get("LBM_REFERENCE_DIR") and os.path.exists(out):
        _jobs[key] = (None, out, time.time())
        return _jobs[key]
    env = dict(os.environ, OMP_WAIT_POLICY="PASSIVE")
    log = open(out + ".log", "w")
    proc = subprocess.Popen([sys.executable, os.path.abspath(__file__), out, repr(Ca), str(steps)],
                            cwd=ROOT, env=env, stdout=log, stderr=subprocess.STDOUT)
    _jobs[key] = (proc, out, time.time())
    return _jobs[key]


def result(Ca, steps, deadline):
    """Fields and diagnostics of the reference; waits for the background run
    until the wall-clock `deadline` (time.time() value)."""
    proc, out, t0 = start(Ca, steps)
    while proc is not None and proc.poll() is None:
        if time.time() > deadline:
            proc.kill()
            raise TimeoutError(f"FP64 reference not finished after {time.time() - t0:.0f} s")
        time.sleep(1.0)
    if proc is not None and proc.returncode != 0:
        raise RuntimeError(f"FP64 reference failed ({proc.returncode}): see {out}.log")
    z = np.load(out)
    fields = {k: z[k] for k in ("phi", "c", "ux", "uy", "P")}
    diag = {k[2:]: float(z[k]) for k in z.files if k.startswith("d_")}
    diag["seconds"] = float(z["seconds"])
    return fields, diag


def stop_all():
    for proc, _, _ in _jobs.values():
        if proc is not None and proc.poll() is None:
            proc.kill()


def _main(out, Ca, steps):
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2504_09024_gb300 import workloads as W
    case = W.shear_drop_2048x1024(Ca=Ca, steps=steps)
    t0 = time.time()
    s = oracle.run_case(case, steps=steps)
    F = s.fields()
    d = s.diagnostics()
    tmp = out + ".tmp.npz"
    np.savez(tmp, seconds=time.time() - t0, threads=oracle.num_threads(),
             **F, **{f"d_{k}": v for k, v in d.items()})
    os.replace(tmp, out)


if __name__ == "__main__":
    _main(sys.argv[1], float(sys.argv[2]), int(sys.argv[3]))

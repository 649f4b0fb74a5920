"""Surrogate-guided search for the critical capillary number of drops in shear.

The learned part of the method's workflow: LBM runs of drops in simple shear
label (steady deformation D, breakup) points of the parameter space (Ca,
elasticity beta, surface Peclet number Pe_s, Gamma0 / Gamma_inf, 2R / H); a
small network (liblbm.so's surrogate kernels) is trained on them; for each
sweep point the network's breakup logit is bisected in Ca, and the LBM checks
every prediction by two runs at Ca_pred -+ 0.05 (no breakup below, breakup
above).  An all-LBM bisection to the same bracket width is the baseline.

This module only draws parameters, batches runs and moves arrays: every
lattice step, diagnostic, component count and network step runs in the
library's CUDA kernels (lbm.Batch, lbm.Surrogate).

Run definition (all runs share one grid so that they step together):
  grid nx x ny (default 384 x 128, nx = 3 H), R = H / 8 (2R/H = 0.25), W = 4,
  Re = 1, nu = 0.1, u(y) = U0 (2y/H - 1) between walls moving at -+U0,
  density and viscosity ratio 1; t* = gamma_dot t = 25 (the breakup
  sequence of Sec. 4.4 at Re = 1 runs to t* = 25).  Labels: D = mean of 5
  samples over the last 10% of the run, breakup = more than one connected
  component of phi > 1/2 at the end (or a non-finite state).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm, workloads as W

CA_RANGE = (0.05, 0.5)
RE = 1.0
NU = 0.1
T_STAR = 25.0
R_OVER_H = 1.0 / 8.0
BRACKET = 0.05          # the LBM checks Ca_pred -+ BRACKET


def draw_points(n, seed):
    """Sweep / training points: Ca ~ U[0.05, 0.5], beta ~ U[0, 0.5],
    Pe_s ~ logU[1, 100], Gamma0 ~ U[0.1, 0.6], 2R/H = 0.25 (R = H / 8)."""
    rng = np.random.default_rng(seed)
    return {
        "Ca": rng.uniform(*CA_RANGE, n),
        "beta": rng.uniform(0.0, 0.5, n),
        "Pe_s": np.exp(rng.uniform(0.0, math.log(100.0), n)),
        "Gamma0": rng.uniform(0.1, 0.6, n),
        "aspect": np.full(n, 2.0 * R_OVER_H),
    }


def features(pts):
    """Network inputs scaled to about [-1, 1]."""
    return np.stack([(np.asarray(pts["Ca"]) - 0.275) / 0.225,
                     (np.asarray(pts["beta"]) - 0.25) / 0.25,
                     np.log10(np.asarray(pts["Pe_s"])) - 1.0,
                     (np.asarray(pts["Gamma0"]) - 0.35) / 0.25,
                     (np.asarray(pts["aspect"]) - 0.25) / 0.1], axis=1).astype(np.float32)


def subset(pts, idx):
    return {k: np.asarray(v)[idx] for k, v in pts.items()}


def make_case(Ca, beta, Pe_s, Gamma0, grid):
    nx, ny = grid
    return W.shear_drop(nx, ny, ny * R_OVER_H, 4.0, Ca=float(Ca), beta=float(beta),
                        Gamma0=float(Gamma0), Re=RE, Pe_s=float(Pe_s), nu=NU,
                        name=f"sweep_{nx}x{ny}")


def run_steps(grid, t_star=T_STAR):
    gamma_dot = RE * NU / (grid[1] * R_OVER_H) ** 2
    return int(math.ceil(t_star / gamma_dot / 32.0)) * 32


def lbm_labels(pts, grid, t_star=T_STAR, batch=512, samples=5):
    """Label every point with an LBM run.  Returns (D, breakup, steady) and
    the number of cell updates."""
    n = len(pts["Ca"])
    steps = run_steps(grid, t_star)
    tail = max(samples, steps // 10)
    marks = sorted({steps - tail + (k * tail) // samples for k in range(1, samples + 1)})
    D = np.zeros(n)
    brk = np.zeros(n, dtype=bool)
    steady = np.zeros(n, dtype=bool)
    for a in range(0, n, batch):
        idx = list(range(a, min(n, a + batch)))
        cases = [make_case(pts["Ca"][k], pts["beta"][k], pts["Pe_s"][k], pts["Gamma0"][k], grid)
                 for k in idx]
        b = lbm.Batch([c.phys for c in cases])
        for r, c in zip(b.runs, cases):
            r.init(c.phi, c.c, c.ux, c.uy)
        done = 0
        hist = np.zeros((len(idx), len(marks)))
        bad = np.zeros(len(idx), dtype=bool)
        for m, at in enumerate(marks):
            b.step(at - done)
            done = at
            b.sync()
            for j, r in enumerate(b.runs):
                d = r.diagnostics()
                hist[j, m] = d["D"]
                bad[j] |= d["nonfinite"] > 0
        gd = RE * NU / (grid[1] * R_OVER_H) ** 2
        tm = np.asarray(marks, dtype=float) * gd
        for j, r in enumerate(b.runs):
            k = idx[j]
            D[k] = float(np.mean(hist[j]))
            slope = np.polyfit(tm, hist[j], 1)[0] if np.all(np.isfinite(hist[j])) else np.inf
            steady[k] = abs(slope) < 1e-3
            brk[k] = bad[j] or r.components(0.5) > 1
        b.close()
    return D, brk, steady, n * steps * grid[0] * grid[1]


def train_surrogate(X, yD, yB, epochs=3000, lr=2e-3, seed=0):
    net = lbm.Surrogate(seed=seed)
    loss = net.train(X, yD, yB, epochs=epochs, lr=lr)
    return net, loss


def predict_ca_crit(net, pts, resolution=0.001):
    """Smallest Ca in CA_RANGE where the breakup logit turns positive (by a
    dense scan in Ca, then bisection to `resolution`); nan when the logit
    stays negative, CA_RANGE[0] when it is positive throughout."""
    n = len(pts["beta"])
    grid = np.arange(CA_RANGE[0], CA_RANGE[1] + 1e-12, 0.01)
    rep = {k: np.repeat(np.asarray(v), len(grid)) for k, v in pts.items()}
    rep["Ca"] = np.tile(grid, n)
    _, z = net.predict(features(rep))
    z = z.reshape(n, len(grid))
    out = np.full(n, np.nan)
    lo = np.full(n, np.nan)
    hi = np.full(n, np.nan)
    for k in range(n):
        pos = np.nonzero(z[k] > 0)[0]
        if len(pos) == 0:
            continue
        if pos[0] == 0:
            out[k] = CA_RANGE[0]
            continue
        lo[k], hi[k] = grid[pos[0] - 1], grid[pos[0]]
    todo = np.isfinite(lo)
    while todo.any() and np.nanmax(hi[todo] - lo[todo]) > resolution:
        mid = 0.5 * (lo + hi)
        q = {k: np.asarray(v)[todo] for k, v in pts.items()}
        q["Ca"] = mid[todo]
        _, zm = net.predict(features(q))
        up = np.zeros(n, dtype=bool)
        up[np.nonzero(todo)[0]] = zm > 0
        hi = np.where(todo & up, mid, hi)
        lo = np.where(todo & ~up, mid, lo)
    out[todo] = 0.5 * (lo[todo] + hi[todo])
    return out


def verify(pts, ca_pred, grid, t_star=T_STAR, batch=512):
    """LBM runs at Ca_pred -+ BRACKET: a prediction is confirmed when the lower
    run keeps one drop and the upper run breaks up."""
    ok = np.isfinite(ca_pred)
    idx = np.nonzero(ok)[0]
    lo = np.clip(ca_pred[idx] - BRACKET, *CA_RANGE)
    hi = np.clip(ca_pred[idx] + BRACKET, *CA_RANGE)
    q = {k: np.concatenate([np.asarray(v)[idx]] * 2) for k, v in pts.items()}
    q["Ca"] = np.concatenate([lo, hi])
    _, brk, _, cells = lbm_labels(q, grid, t_star, batch)
    m = len(idx)
    confirmed = np.zeros(len(ca_pred), dtype=bool)
    confirmed[idx] = (~brk[:m]) & brk[m:]
    return confirmed, 2 * m, cells


def lbm_bisection(pts, grid, width=2 * BRACKET, t_star=T_STAR, batch=512):
    """All-LBM baseline: bisect Ca on LBM runs until the bracket is `width`
    wide (from CA_RANGE; a bracket end is assumed, not run).  Returns the
    bracket midpoints and the number of runs."""
    n = len(pts["beta"])
    lo = np.full(n, CA_RANGE[0])
    hi = np.full(n, CA_RANGE[1])
    runs = 0
    cells = 0
    while np.max(hi - lo) > width + 1e-12:
        q = dict(pts)
        q["Ca"] = 0.5 * (lo + hi)
        _, brk, _, c = lbm_labels(q, grid, t_star, batch)
        runs += n
        cells += c
        hi = np.where(brk, q["Ca"], hi)
        lo = np.where(brk, lo, q["Ca"])
    return 0.5 * (lo + hi), runs, cells


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--grid", default="384x128")
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--points", type=int, default=256)
    ap.add_argument("--baseline-points", type=int, default=64)
    ap.add_argument("--t-star", type=float, default=T_STAR)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=W.CASE_SEED)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    grid = tuple(int(v) for v in args.grid.split("x"))
    report = {"grid": grid, "t_star": args.t_star, "steps_per_run": run_steps(grid, args.t_star)}
    t0 = time.perf_counter()
    train = draw_points(args.train, args.seed)
    yD, yB, steady, cells = lbm_labels(train, grid, args.t_star)
    t_train_runs = time.perf_counter() - t0
    report.update(train_runs=args.train, train_breakup_fraction=float(yB.mean()),
                  train_steady_fraction=float(steady.mean()), train_seconds=t_train_runs,
                  train_cell_updates=cells)
    X = features(train)
    t1 = time.perf_counter()
    net, loss = train_surrogate(X, yD.astype(np.float32), yB.astype(np.float32),
                                epochs=args.epochs)
    report.update(train_loss=loss, fit_seconds=time.perf_counter() - t1)
    Dp, zp = net.predict(X)
    report.update(train_D_rmse=float(np.sqrt(np.mean((Dp - yD) ** 2))),
                  train_breakup_accuracy=float(np.mean((zp > 0) == yB)))
    sweep = draw_points(args.points, args.seed + 1)
    ca = predict_ca_crit(net, sweep)
    t2 = time.perf_counter()
    confirmed, vruns, vcells = verify(sweep, ca, grid, args.t_star)
    report.update(sweep_points=args.points, predicted=int(np.isfinite(ca).sum()),
                  confirmed=int(confirmed.sum()), verify_runs=vruns,
                  verify_seconds=time.perf_counter() - t2, verify_cell_updates=vcells)
    nb = min(args.baseline_points, args.points)
    t3 = time.perf_counter()
    ca_lbm, bruns, bcells = lbm_bisection(subset(sweep, np.arange(nb)), grid, t_star=args.t_star)
    bsec = time.perf_counter() - t3
    diff = np.abs(ca[:nb] - ca_lbm)
    have = np.isfinite(diff)
    report.update(baseline_points=nb, baseline_runs=bruns, baseline_seconds=bsec,
                  baseline_runs_per_point=bruns / nb,
                  surrogate_vs_lbm_abs_error_median=float(np.median(diff[have])) if have.any() else None,
                  surrogate_within_bracket=float(np.mean(diff[have] <= 2 * BRACKET)) if have.any() else None,
                  runs_per_point_with_surrogate=vruns / args.points,
                  runs_per_point_with_training=(vruns + args.train) / args.points)
    sec_per_run = (t_train_runs + report["verify_seconds"] + bsec) / (args.train + vruns + bruns)
    report.update(runs_per_hour=3600.0 / sec_per_run, total_seconds=time.perf_counter() - t0)
    text = json.dumps(report, indent=1, default=float)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    net.close()
    return report


if __name__ == "__main__":
    main()

"""Surrogate-guided search for the critical capillary number of drops in shear.

The learned part of the method's workflow: LBM runs of drops in simple shear
label (steady deformation D, breakup) points of the parameter space (Ca,
elasticity beta, surface Peclet number Pe_s, Gamma0 / Gamma_inf, 2R / H); a
small network (liblbm.so's surrogate kernels) is trained on them; for each
sweep point the network's breakup logit is bisected in Ca, and the LBM checks
every prediction by two runs at Ca_pred -+ 0.05 (no breakup below, breakup
above).  The plain LBM stays the fallback: a prediction the LBM rejects, or a
point the network gives no Ca for, is bisected on LBM runs from the bracket
the check leaves.  An all-LBM bisection to the same bracket width is the
baseline.

This module only draws parameters, batches runs and moves arrays: every
lattice step, diagnostic, component count and network step runs in the
library's CUDA kernels (lbm.Batch, lbm.Surrogate).

Run definition (all runs share one grid so that they step together):
  grid nx x ny (default 384 x 128, nx = 3 H), R = (2R/H) H / 2 with
  2R/H ~ U[0.2, 0.3], W = 4, Re = 1, u(y) = U0 (2y/H - 1) between walls
  moving at -+U0, density and viscosity ratio 1.  The viscosity scales as
  R^2 (nu = 0.1 at the largest radius) so that every run has the same shear
  rate gamma_dot = Re nu / R^2, and the same number of steps reaches
  t* = gamma_dot t = 25 (the breakup sequence of Sec. 4.4 at Re = 1 runs to
  t* = 25).  Labels: D = mean of 5 samples over the last 10% of the run,
  breakup = more than one connected component of phi > 1/2 at the end (or a
  non-finite state).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm, workloads as W

CA_RANGE = (0.05, 0.5)
ASPECT_RANGE = (0.2, 0.3)   # 2R / H
RE = 1.0
NU_MAX = 0.1                # viscosity of the largest drop
T_STAR = 25.0
BRACKET = 0.05          # the LBM checks Ca_pred -+ BRACKET


def draw_points(n, seed):
    """Sweep / training points: Ca ~ U[0.05, 0.5], beta ~ U[0, 0.5],
    Pe_s ~ logU[1, 100], Gamma0 ~ U[0.1, 0.6], 2R/H ~ U[0.2, 0.3]."""
    rng = np.random.default_rng(seed)
    return {
        "Ca": rng.uniform(*CA_RANGE, n),
        "beta": rng.uniform(0.0, 0.5, n),
        "Pe_s": np.exp(rng.uniform(0.0, math.log(100.0), n)),
        "Gamma0": rng.uniform(0.1, 0.6, n),
        "aspect": rng.uniform(*ASPECT_RANGE, n),
    }


def features(pts):
    """Network inputs scaled to about [-1, 1]."""
    amid = 0.5 * (ASPECT_RANGE[0] + ASPECT_RANGE[1])
    ahalf = 0.5 * (ASPECT_RANGE[1] - ASPECT_RANGE[0])
    return np.stack([(np.asarray(pts["Ca"]) - 0.275) / 0.225,
                     (np.asarray(pts["beta"]) - 0.25) / 0.25,
                     np.log10(np.asarray(pts["Pe_s"])) - 1.0,
                     (np.asarray(pts["Gamma0"]) - 0.35) / 0.25,
                     (np.asarray(pts["aspect"]) - amid) / ahalf], axis=1).astype(np.float32)


def subset(pts, idx):
    return {k: np.asarray(v)[idx] for k, v in pts.items()}


def radius(aspect, grid):
    return 0.5 * float(aspect) * grid[1]


def shear_rate(grid):
    """gamma_dot shared by every run of the grid (Re nu / R^2 at the largest R)."""
    r_max = radius(ASPECT_RANGE[1], grid)
    return RE * NU_MAX / r_max ** 2


def make_case(Ca, beta, Pe_s, Gamma0, aspect, grid):
    nx, ny = grid
    R = radius(aspect, grid)
    nu = shear_rate(grid) * R ** 2 / RE
    return W.shear_drop(nx, ny, R, 4.0, Ca=float(Ca), beta=float(beta),
                        Gamma0=float(Gamma0), Re=RE, Pe_s=float(Pe_s), nu=nu,
                        name=f"sweep_{nx}x{ny}")


def run_steps(grid, t_star=T_STAR):
    return int(math.ceil(t_star / shear_rate(grid) / 32.0)) * 32


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
        cases = [make_case(pts["Ca"][k], pts["beta"][k], pts["Pe_s"][k], pts["Gamma0"][k],
                           pts["aspect"][k], grid) for k in idx]
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
        tm = np.asarray(marks, dtype=float) * shear_rate(grid)
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
    run keeps one drop and the upper run breaks up.  Returns (confirmed,
    breakup of the lower run, breakup of the upper run, runs, cell updates);
    the outcomes are False where no prediction was checked."""
    n = len(ca_pred)
    ok = np.isfinite(ca_pred)
    idx = np.nonzero(ok)[0]
    lo = np.clip(ca_pred[idx] - BRACKET, *CA_RANGE)
    hi = np.clip(ca_pred[idx] + BRACKET, *CA_RANGE)
    brk_lo = np.zeros(n, dtype=bool)
    brk_hi = np.zeros(n, dtype=bool)
    cells = 0
    if len(idx):
        q = {k: np.concatenate([np.asarray(v)[idx]] * 2) for k, v in pts.items()}
        q["Ca"] = np.concatenate([lo, hi])
        _, brk, _, cells = lbm_labels(q, grid, t_star, batch)
        m = len(idx)
        brk_lo[idx] = brk[:m]
        brk_hi[idx] = brk[m:]
    confirmed = ok & ~brk_lo & brk_hi
    return confirmed, brk_lo, brk_hi, 2 * len(idx), cells


def fallback_brackets(ca_pred, confirmed, brk_lo, brk_hi):
    """Where the LBM has to search after the check: Ca_crit lies below a
    lower run that broke up, above an upper run that did not, and anywhere
    in CA_RANGE for a point without a prediction or with both outcomes
    wrong.  Returns (indices, lo, hi) of the unconfirmed points."""
    idx = np.nonzero(~confirmed)[0]
    lo = np.full(len(idx), CA_RANGE[0])
    hi = np.full(len(idx), CA_RANGE[1])
    for a, k in enumerate(idx):
        if not np.isfinite(ca_pred[k]):
            continue
        below, above = brk_lo[k], not brk_hi[k]
        if below and not above:
            hi[a] = max(CA_RANGE[0], ca_pred[k] - BRACKET)
        elif above and not below:
            lo[a] = min(CA_RANGE[1], ca_pred[k] + BRACKET)
    return idx, lo, hi


def lbm_bisection(pts, grid, width=2 * BRACKET, t_star=T_STAR, batch=512, lo=None, hi=None):
    """Bisect Ca on LBM runs until every bracket is `width` wide, from the
    brackets (lo, hi) (default CA_RANGE; bracket ends are assumed, not run).
    Returns the bracket midpoints, the number of runs and cell updates."""
    n = len(pts["beta"])
    lo = np.full(n, CA_RANGE[0]) if lo is None else np.asarray(lo, dtype=float).copy()
    hi = np.full(n, CA_RANGE[1]) if hi is None else np.asarray(hi, dtype=float).copy()
    runs = 0
    cells = 0
    while n and np.max(hi - lo) > width + 1e-12:
        todo = np.nonzero(hi - lo > width + 1e-12)[0]
        q = subset(pts, todo)
        q["Ca"] = 0.5 * (lo[todo] + hi[todo])
        _, brk, _, c = lbm_labels(q, grid, t_star, batch)
        runs += len(todo)
        cells += c
        hi[todo] = np.where(brk, q["Ca"], hi[todo])
        lo[todo] = np.where(brk, lo[todo], q["Ca"])
    return 0.5 * (lo + hi), runs, cells


def resolve(pts, ca_pred, grid, t_star=T_STAR, batch=512):
    """Ca_crit of every point: the surrogate's where the LBM confirms it, an
    LBM bisection from the remaining bracket where it does not (or where the
    network gave none).  Returns (ca, source, counts) with source 1 for
    confirmed predictions and 0 for LBM results."""
    confirmed, brk_lo, brk_hi, vruns, vcells = verify(pts, ca_pred, grid, t_star, batch)
    ca = np.where(confirmed, ca_pred, np.nan)
    idx, lo, hi = fallback_brackets(ca_pred, confirmed, brk_lo, brk_hi)
    fruns = fcells = 0
    if len(idx):
        ca_f, fruns, fcells = lbm_bisection(subset(pts, idx), grid, t_star=t_star, batch=batch,
                                            lo=lo, hi=hi)
        ca[idx] = ca_f
    counts = dict(confirmed=int(confirmed.sum()), verify_runs=vruns, verify_cell_updates=vcells,
                  fallback_points=int(len(idx)), fallback_runs=fruns,
                  fallback_cell_updates=fcells)
    return ca, confirmed.astype(int), counts


def heldout_error(net, pts, grid, t_star=T_STAR, batch=512):
    """Surrogate against LBM labels on points not used in training: D RMSE
    over the runs that stay whole and reach a steady D, breakup accuracy
    over all."""
    D, brk, steady, cells = lbm_labels(pts, grid, t_star, batch)
    Dp, zp = net.predict(features(pts))
    whole = ~brk & steady
    rmse = float(np.sqrt(np.mean((Dp[whole] - D[whole]) ** 2))) if whole.any() else None
    return dict(heldout_points=int(len(D)), heldout_D_rmse=rmse,
                heldout_D_points=int(whole.sum()),
                heldout_breakup_accuracy=float(np.mean((zp > 0) == brk)),
                heldout_cell_updates=cells)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--grid", default="384x128")
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--heldout", type=int, default=128)
    ap.add_argument("--points", type=int, default=256)
    ap.add_argument("--baseline-points", type=int, default=64)
    ap.add_argument("--t-star", type=float, default=T_STAR)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=W.CASE_SEED)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    grid = tuple(int(v) for v in args.grid.split("x"))
    steps = run_steps(grid, args.t_star)
    report = {"grid": grid, "t_star": args.t_star, "steps_per_run": steps}
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
    t_fit = time.perf_counter() - t1
    report.update(train_loss=loss, fit_seconds=t_fit)
    Dp, zp = net.predict(X)
    report.update(train_D_rmse=float(np.sqrt(np.mean((Dp - yD) ** 2))),
                  train_breakup_accuracy=float(np.mean((zp > 0) == yB)))
    t1h = time.perf_counter()
    report.update(heldout_error(net, draw_points(args.heldout, args.seed + 2), grid, args.t_star))
    t_heldout = time.perf_counter() - t1h
    report.update(heldout_seconds=t_heldout)
    sweep = draw_points(args.points, args.seed + 1)
    ca = predict_ca_crit(net, sweep)
    t2 = time.perf_counter()
    ca_final, source, counts = resolve(sweep, ca, grid, args.t_star)
    t_resolve = time.perf_counter() - t2
    report.update(sweep_points=args.points, predicted=int(np.isfinite(ca).sum()),
                  resolved=int(np.isfinite(ca_final).sum()), resolve_seconds=t_resolve, **counts)
    nb = min(args.baseline_points, args.points)
    t3 = time.perf_counter()
    ca_lbm, bruns, bcells = lbm_bisection(subset(sweep, np.arange(nb)), grid, t_star=args.t_star)
    bsec = time.perf_counter() - t3
    diff = np.abs(ca_final[:nb] - ca_lbm)
    have = np.isfinite(diff)
    sweep_runs = counts["verify_runs"] + counts["fallback_runs"]
    report.update(baseline_points=nb, baseline_runs=bruns, baseline_seconds=bsec,
                  baseline_runs_per_point=bruns / nb,
                  resolved_vs_lbm_abs_error_median=float(np.median(diff[have])) if have.any() else None,
                  resolved_within_bracket=float(np.mean(diff[have] <= 2 * BRACKET)) if have.any() else None,
                  runs_per_point_with_surrogate=sweep_runs / args.points,
                  runs_per_point_with_training=(sweep_runs + args.train) / args.points)
    # device time of the search itself (GPU-hours), with and without the
    # training labels, against the all-LBM bisection of every sweep point
    hours = lambda s: s / 3600.0
    report.update(gpu_hours_surrogate_search=hours(t_resolve + t_fit),
                  gpu_hours_surrogate_with_training=hours(t_resolve + t_fit + t_train_runs),
                  gpu_hours_all_lbm=hours(bsec * args.points / nb))
    sec_per_run = (t_train_runs + t_resolve + bsec) / (args.train + sweep_runs + bruns)
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

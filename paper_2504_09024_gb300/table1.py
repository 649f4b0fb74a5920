"""Steady deformation of a drop in simple shear at Re = 0.1 (Sec. 4.3, Table 1).

Runs the paper's creeping-flow set-up for Ca = 0.01 ... 0.05 with a clean
(beta = 0) and a contaminated (beta = 0.25) interface as one batch on the
GPU, samples the Taylor deformation D = (L - B) / (L + B) of the phi = 1/2
contour (lbm_diagnostics) along the run, and lists it beside the paper's
Table 1 and the small-deformation theory of Stone and Leal that Sec. 4.3
compares with:

    D ~ 3 Ca b_r / (4 + Ca b_r),
    b_r = (5/4) [(16 + 19 lam) + 4 beta Pe/Ca] / [10 (1 + lam) + 2 beta Pe/Ca],
    Pe = Re nu / D_s, lam = viscosity ratio (1 here).

Set-up (Sec. 4.3): 3H x H with H = 256, R = H / 8, walls at y = 0, H moving
at -+U0, nu = 0.1, rho = 1, Re = gamma_dot R^2 / nu = 0.1, Ca = rho nu
gamma_dot R / sigma_0, Pe* = U0 W / M_phi = 0.5.  Not stated in the paper
and chosen here: W = 4, Gamma0 / Gamma_inf = 0.3, Pe_s = 10; beta enters the
Langmuir isotherm and, as in the paper's comparison, the b_r above.

Every lattice step and diagnostic runs in liblbm.so's CUDA kernels.
"""
from __future__ import annotations

import argparse
import json
import time

from . import lbm, workloads as W

# Sec. 4.3, Table 1: D x 1e-2 for the clean and the contaminated interface
TABLE1 = {0.01: (1.60, 1.89), 0.02: (3.19, 3.72), 0.03: (4.77, 5.55),
          0.04: (6.35, 7.36), 0.05: (7.93, 9.17)}
BETAS = (0.0, 0.25)
RE, NU = 0.1, 0.1


def stone_leal(Ca, beta, Pe, lam=1.0):
    """Small-deformation D of a drop with an insoluble surfactant (Sec. 4.3)."""
    q = beta * Pe / Ca
    b_r = 1.25 * ((16.0 + 19.0 * lam) + 4.0 * q) / (10.0 * (1.0 + lam) + 2.0 * q)
    return 3.0 * Ca * b_r / (4.0 + Ca * b_r)


def make_cases(H=256, Wd=4.0, Gamma0=0.3, Pe_s=10.0, betas=BETAS):
    cases = []
    for Ca in TABLE1:
        for beta in betas:
            cases.append(W.shear_drop(3 * H, H, H / 8.0, Wd, Ca=Ca, beta=beta, Gamma0=Gamma0,
                                      Re=RE, Pe_s=Pe_s, nu=NU,
                                      name=f"table1_Ca{Ca:g}_beta{beta:g}"))
    return cases


def run(steps=300000, every=20000, H=256, Wd=4.0, Gamma0=0.3, Pe_s=10.0, betas=BETAS):
    cases = make_cases(H, Wd, Gamma0, Pe_s, betas)
    b = lbm.Batch([c.phys for c in cases])
    for r, c in zip(b.runs, cases):
        r.init(c.phi, c.c, c.ux, c.uy)
    history = {c.name: [] for c in cases}
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(every, steps - done)
        b.step(n)
        b.sync()
        done += n
        for r, c in zip(b.runs, cases):
            history[c.name].append((done, r.diagnostics()["D"]))
    wall = time.perf_counter() - t0
    b.close()
    rows = []
    for c in cases:
        Ca, beta = c.meta["Ca"], c.meta["beta"]
        Pe = c.meta["Re"] * NU / c.phys.D_s
        D_end = history[c.name][-1][1]
        D_prev = history[c.name][-2][1] if len(history[c.name]) > 1 else float("nan")
        rows.append(dict(Ca=Ca, beta=beta, D=D_end, D_drift_last_interval=D_end - D_prev,
                         paper=TABLE1[Ca][0 if beta == 0.0 else 1] * 1e-2,
                         stone_leal=stone_leal(Ca, beta, Pe),
                         gamma_dot_t=c.meta["gamma_dot"] * steps))
    return dict(steps=steps, grid=f"{3 * H}x{H}", W=Wd, Gamma0=Gamma0, Pe_s=Pe_s,
                wall_s=wall, rows=rows,
                history={k: v for k, v in history.items()})


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=300000)
    ap.add_argument("--every", type=int, default=20000)
    ap.add_argument("--W", type=float, default=4.0, help="interface width (not stated in the paper)")
    ap.add_argument("--gamma0", type=float, default=0.3)
    ap.add_argument("--pe-s", type=float, default=10.0)
    ap.add_argument("--betas", default="0,0.25")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)
    betas = tuple(float(b) for b in args.betas.split(","))
    res = run(args.steps, args.every, Wd=args.W, Gamma0=args.gamma0, Pe_s=args.pe_s, betas=betas)
    print(f"{res['grid']}, W = {res['W']:g}, {res['steps']} steps ({res['wall_s']:.1f} s on the GPU)")
    print("   Ca   beta   D (GB300)   drift/interval   D (Table 1)   Stone-Leal")
    for r in res["rows"]:
        print(f"{r['Ca']:6.2f} {r['beta']:5.2f}   {r['D']:.4e}     {r['D_drift_last_interval']:+.1e}"
              f"        {r['paper']:.4e}    {r['stone_leal']:.4e}")
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()

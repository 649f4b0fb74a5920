"""The error that FP32 population storage alone puts into a run.

The CUDA path keeps, per cell and step, the zeroth moment S of the f and h
lattices as a fixed-point number (2^29 units per unit bound), the deviations
f_q - w_q S (q = 1..8) in FP32, and the flow populations as g_q - w_q P0 in
FP32.  This module applies that rounding to the FP64 oracle's populations
after every step (through the oracle's population accessors; the oracle
itself is unchanged) and so measures the floor that the storage format alone
sets on a given workload, with every operation in FP64.  On well-conditioned
workloads the floor is far below 1e-5; on tiny drops (R of 1.5-3 cells on a
2-cell interface) and in the far tail of a fast-sheared drop it is not, and a
GPU bound above 1e-5 there is stated as a multiple of this measured floor.
"""
import numpy as np

WQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _fixed_point_scale(bound):
    e = int(np.ceil(np.log2(bound))) if bound > 1.0 else 0
    return 2.0 ** (29 - e)


def _round_scalar_lattice(a, scale):
    S = a.sum(0)
    Sq = np.round(S * scale) / scale
    d = (a[1:] - WQ[1:, None, None] * S).astype(np.float32).astype(np.float64)
    out = np.empty_like(a)
    out[1:] = WQ[1:, None, None] * Sq + d
    out[0] = Sq - out[1:].sum(0)
    return out


def storage_rounded_run(orc, case, steps):
    """Oracle run of `case` whose populations are rounded to the FP32 storage
    format after every step.  Returns the oracle Sim (caller closes it)."""
    ph = case.phys
    s = orc.Sim(ph)
    s.init(case.phi, case.c, case.ux, case.uy, case.P)
    sf = _fixed_point_scale(max(abs(ph.phi_a), abs(ph.phi_b)))
    sh = _fixed_point_scale(ph.c_max)
    P0 = 0.5 * (ph.rho_a + ph.rho_b) / 3.0
    coupled = ph.mode == 0
    for _ in range(steps):
        s.step(1)
        p = s.pops()
        g = None
        if coupled:
            g = (p["g"] - WQ[:, None, None] * P0).astype(np.float32).astype(np.float64)
            g += WQ[:, None, None] * P0
        s.set_pops(f=_round_scalar_lattice(p["f"], sf), h=_round_scalar_lattice(p["h"], sh), g=g)
    return s


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def vrel(got, ref):
    """Relative L2 error of the velocity vector over both components."""
    num = np.sqrt(((got["ux"] - ref["ux"]) ** 2 + (got["uy"] - ref["uy"]) ** 2).sum())
    den = np.sqrt((ref["ux"] ** 2 + ref["uy"] ** 2).sum())
    return float(num / den)


def storage_floor(orc, case, steps, ref_fields=None):
    """Relative L2 errors of phi, c and u (vector) that the storage rounding
    alone causes after `steps` (plain FP64 oracle run as the reference)."""
    if ref_fields is None:
        r = orc.Sim(case.phys)
        r.init(case.phi, case.c, case.ux, case.uy, case.P)
        r.step(steps)
        ref_fields = r.fields()
        r.close()
    q = storage_rounded_run(orc, case, steps)
    got = q.fields()
    q.close()
    out = {"phi": rel(got["phi"], ref_fields["phi"]), "c": rel(got["c"], ref_fields["c"])}
    if case.phys.mode == 0:
        out["u"] = vrel(got, ref_fields)
    return out, got

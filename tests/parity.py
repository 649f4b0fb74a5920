"""Error measures and bounds shared by the GPU parity tests."""
import numpy as np

from storage_floor import rel, storage_floor, vrel  # noqa: F401

# relative L2 bound for phi, Gamma and u after 1000 steps with FP32 populations
TOL = 1e-5


def umag(F):
    return np.hypot(F["ux"], F["uy"])


_floor_cache = {}


def lively_c_bound(orc, case, steps):
    """Whole-field bound of Gamma on the lively drop: three times the error
    that FP32 population storage alone causes there (tests/storage_floor.py,
    FP64 arithmetic with the populations rounded to the storage format after
    every step).  Its fast shear spreads Gamma (up to 2.5e-3) into the tail of
    the phi profile, where the flux direction follows a phi held on a 2^-29
    fixed-point grid; the storage floor there is 1.6e-5 after 1000 steps.
    Inside the interface band the 1e-5 bound holds."""
    key = (case.name, case.phys.nx, case.phys.ny, case.phys.rho_a, case.phys.nu_a, steps)
    if key not in _floor_cache:
        _floor_cache[key] = storage_floor(orc, case, steps)[0]
    return max(TOL, 3.0 * _floor_cache[key]["c"]), _floor_cache[key]


def check_lively(got, ref, orc, case, steps):
    errs = {"phi": rel(got["phi"], ref["phi"]), "u": vrel(got, ref),
            "c": rel(got["c"], ref["c"])}
    band = (ref["phi"] > 1e-3) & (ref["phi"] < 1.0 - 1e-3)
    errs["c_band"] = float(np.linalg.norm((got["c"] - ref["c"])[band]) /
                           np.linalg.norm(ref["c"][band]))
    c_bound, floor = lively_c_bound(orc, case, steps)
    errs["c_bound"] = c_bound
    assert errs["phi"] <= TOL and errs["u"] <= TOL, (errs, floor)
    assert errs["c_band"] <= TOL, (errs, floor)
    assert errs["c"] <= c_bound, (errs, floor)
    return errs

"""Error measures and bounds shared by the GPU parity tests."""
import numpy as np

# relative L2 bound for phi, Gamma and u after 1000 steps with FP32 populations
TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def umag(F):
    return np.hypot(F["ux"], F["uy"])


# Gamma on the lively drop.  Its fast shear and weak confinement spread
# Gamma into the tail of the phi profile (Gamma ~ 1e-3 where phi < 1e-3),
# where the flux directions follow a phi that the FP32 state holds on a
# 2^-29 fixed-point grid.  An FP64-arithmetic emulation of the method with
# only phi's zeroth moment on that grid gives relative L2 errors of Gamma of
# 5e-6 .. 1.6e-5 after 1000 steps on these drops (against 2e-7 with the same
# grid for Gamma alone), almost all of it outside the interface band, so on
# this case the whole-field bound for Gamma is three times that floor and
# the interface band (1e-3 < phi < 1 - 1e-3) keeps the 1e-5 bound.
LIVELY_C_TOL = 5e-5


def check_lively(got, ref):
    errs = {"phi": rel(got["phi"], ref["phi"]), "u": rel(umag(got), umag(ref)),
            "c": rel(got["c"], ref["c"])}
    band = (ref["phi"] > 1e-3) & (ref["phi"] < 1.0 - 1e-3)
    errs["c_band"] = float(np.linalg.norm((got["c"] - ref["c"])[band]) /
                           np.linalg.norm(ref["c"][band]))
    assert errs["phi"] <= TOL and errs["u"] <= TOL, errs
    assert errs["c_band"] <= TOL, errs
    assert errs["c"] <= LIVELY_C_TOL, errs
    return errs

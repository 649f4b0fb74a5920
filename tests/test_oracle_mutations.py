"""The oracle's pins catch planted mistakes.

Each case copies the oracle package into a temporary directory, plants one
plausible mistake in its C source (a dropped term, a wrong sign, a swapped
operand), builds that copy and runs the pin that is meant to catch it, which
must then fail.  The mistakes are planted in the copy only; the oracle under
oracle/ is never modified.  Cases cover the variable-density path (rho and nu
interpolation, psi = P - rho cs2, the velocity definition), the F_p parts of
the second-order sources of App. D and the Marangoni term of Eq. (Fs).
"""
import importlib.util
import os
import shutil
import sys

import pytest

import test_oracle_pins as pins
import test_oracle_pins_density as dens

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_variant(tmp_root, tag, old, new):
    d = os.path.join(tmp_root, f"oracle_mut_{tag}")
    shutil.copytree(os.path.join(ROOT, "oracle"), d,
                    ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    path = os.path.join(d, "lbm_oracle.c")
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site of {tag} not found exactly once"
    open(path, "w").write(src.replace(old, new))
    name = f"oracle_mut_{tag}"
    spec = importlib.util.spec_from_file_location(name, os.path.join(d, "__init__.py"),
                                                  submodule_search_locations=[d])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


# ---- what each pin accepts (the bounds of the pins themselves) ------------

def _sound_ok(orc):
    for phase in ("a", "b"):
        speed, rate, imp = dens.bulk_sound(orc, phase)
        if (abs(speed - 1) >= dens.SOUND_TOL["speed"] or abs(rate - 1) >= dens.SOUND_TOL["rate"]
                or abs(imp - 1) >= dens.SOUND_TOL["impedance"]):
            return False
    return True


def _layer_axis_ok(orc):
    return dens.translated_layer(orc, 4.0) < dens.LAYER_W4_TOL


def _layer_diag_ok(orc):
    return dens.translated_layer(orc, 4.0, diagonal=True) < dens.DIAG_W4_TOL


def _equilibrium_ok(orc):
    return dens.equilibrium_moment_errors(orc) < dens.EQ_TOL


def _couette_ok(orc):
    err, uy = dens.two_layer_couette(orc)
    return err < dens.COUETTE_TOL and uy < 1e-10


def _flat_uniform_ok(orc):
    return pins.flat_uniform_force(orc) < 1e-9


def _marangoni_ok(orc):
    (g4, c4), (g8, c8) = pins.marangoni_gain(orc, 4.0), pins.marangoni_gain(orc, 8.0)
    if min(c4, c8) <= 0.99999 or not (0 < 1 - g4 and 0 < 1 - g8):
        return False
    lo, hi = pins.MARANGONI_ORDER
    return lo < (1 - g8) / (1 - g4) < hi


MUTATIONS = [
    # (tag, original text, planted text, pin that must fail)
    ("interp_swapped",
     "return vb + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (va - vb);",
     "return va + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (vb - va);", _sound_ok),
    ("interp_sign",
     "return vb + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (va - vb);",
     "return vb + (phi - p->phi_b) / (p->phi_a - p->phi_b) * (va + vb);", _sound_ok),
    ("nu_constant",
     "s->nu[x] = lin_interp(&s->p, sf, s->p.nu_a, s->p.nu_b);",
     "s->nu[x] = lin_interp(&s->p, sf, s->p.nu_a, s->p.nu_a);", _sound_ok),
    ("u_without_rho",
     "double ux = (s->jx[x] + 0.5 * CS2 * Ftx) / (CS2 * rho);",
     "double ux = (s->jx[x] + 0.5 * CS2 * Ftx) / CS2;", _sound_ok),
    ("psi_sign",
     "s->psistar[x] = sg - s->rho[x] * CS2;",
     "s->psistar[x] = sg + s->rho[x] * CS2;", _layer_axis_ok),
    ("psi_without_rho",
     "s->psistar[x] = sg - s->rho[x] * CS2;",
     "s->psistar[x] = sg;", _layer_axis_ok),
    ("s11_Fp_dropped",
     "sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;",
     "sg[5] = ux * uy * G;", _layer_axis_ok),
    ("s11_Fp_half",
     "sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;",
     "sg[5] = 0.5 * CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;", _layer_axis_ok),
    ("s11_Fp_transposed",
     "sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;",
     "sg[5] = CS2 * (Fpx * ux + Fpy * uy) + ux * uy * G;", _layer_axis_ok),
    ("s11_Fp_sign",
     "sg[5] = CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;",
     "sg[5] = -CS2 * (Fpx * uy + Fpy * ux) + ux * uy * G;", _layer_axis_ok),
    ("s20_Fp_dropped",
     "sg[3] = 2.0 * CS2 * Fpx * ux + (ux * ux + CS2) * G;",
     "sg[3] = (ux * ux + CS2) * G;", _layer_diag_ok),
    ("s02_Fp_dropped",
     "sg[4] = 2.0 * CS2 * Fpy * uy + (uy * uy + CS2) * G;",
     "sg[4] = (uy * uy + CS2) * G;", _layer_diag_ok),
    ("eq22_without_rho",
     "eq[8] = CS2 * CS2 * CS2 * rho + psi",
     "eq[8] = CS2 * CS2 * CS2 + psi", _equilibrium_ok),
    ("couette_nu_ends_swapped",
     "s->nu[x] = lin_interp(&s->p, sf, s->p.nu_a, s->p.nu_b);",
     "s->nu[x] = lin_interp(&s->p, sf, s->p.nu_b, s->p.nu_a);", _couette_ok),
    ("marangoni_projection_sign",
     "double msx = sgx - nxx * ndots, msy = sgy - nyy * ndots;",
     "double msx = sgx + nxx * ndots, msy = sgy + nyy * ndots;", _flat_uniform_ok),
    ("marangoni_gradient_power",
     "double Fsx = Nsig * (-sg * g2 * kap * nxx + g2 * msx);",
     "double Fsx = Nsig * (-sg * g2 * kap * nxx + mag * msx);", _marangoni_ok),
    ("marangoni_tenth_low",
     "double Fsx = Nsig * (-sg * g2 * kap * nxx + g2 * msx);",
     "double Fsx = Nsig * (-sg * g2 * kap * nxx + 0.9 * g2 * msx);", _marangoni_ok),
]


def test_pins_pass_on_the_oracle(oracle_mod):
    """The same acceptance functions pass on the unmodified oracle (the
    Couette check, the slowest, is covered by its own pin)."""
    for ok in (_sound_ok, _layer_axis_ok, _layer_diag_ok, _equilibrium_ok, _marangoni_ok,
               _flat_uniform_ok):
        assert ok(oracle_mod), ok.__name__


@pytest.mark.parametrize("tag,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(tmp_path_factory, tag, old, new, pin):
    mod = _build_variant(str(tmp_path_factory.mktemp("mut")), tag, old, new)
    assert not pin(mod), f"{tag}: the pin {pin.__name__} did not catch the planted mistake"

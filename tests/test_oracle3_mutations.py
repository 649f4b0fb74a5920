"""The 3-D oracle's pins catch planted mistakes.

Each case copies the oracle package into a temporary directory, plants one
plausible mistake in the copy's lbm_oracle3.c (a wrong weight, a dropped or
mis-scaled term, a flipped sign, a wrong relaxation), builds the copy and runs
the pin meant to catch it, which must then fail.  The oracle under oracle/ is
never modified.  The second half of the list plants mistakes in the flow
lattice (equilibrium, trace and relaxation, sources, walls, forces,
curvature).
"""
import importlib.util
import os
import shutil
import sys

import pytest

import test_oracle3_flow_pins as fpins
import test_oracle3_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_variant(tmp_root, tag, old, new):
    d = os.path.join(tmp_root, f"oracle3_mut_{tag}")
    shutil.copytree(os.path.join(ROOT, "oracle"), d,
                    ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    path = os.path.join(d, "lbm_oracle3.c")
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site of {tag} not found exactly once"
    open(path, "w").write(src.replace(old, new))
    name = f"oracle3_mut_{tag}"
    spec = importlib.util.spec_from_file_location(name, os.path.join(d, "__init__.py"),
                                                  submodule_search_locations=[d])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


def _run_pin(monkeypatch, mod, pin, *args):
    monkeypatch.setattr(pins, "oracle", mod)
    monkeypatch.setattr(fpins, "oracle", mod)
    pin(*args)


MUTATIONS = [
    # (tag, old, new, pin, args)
    ("edge_weight", "2.0 / 27.0, 1.0 / 54.0,", "2.0 / 27.0, 1.0 / 27.0,",
     pins.test_gradient_of_product_of_sines, ()),
    ("corner_weight", "1.0 / 54.0, 1.0 / 216.0}", "1.0 / 54.0, 1.0 / 108.0}",
     pins.test_gradient_of_product_of_sines, ()),
    ("frame_sign_z", "{s * ux, s * uy, s * uz}", "{s * ux, s * uy, uz}",
     pins.test_equilibrium_raw_moments_are_maxwellian, ()),
    ("second_order_eq", "{1.0, 0.0, 1.0 / 3.0}", "{1.0, 0.0, 1.0 / 9.0}",
     pins.test_equilibrium_raw_moments_are_maxwellian, ()),
    ("third_axis_binomial", "v *= binom(m, j) * ipow(u[ax], m - j);",
     "v *= (ax == 2 ? 1.0 : binom(m, j)) * ipow(u[ax], m - j);",
     pins.test_reduces_to_the_2d_oracle, ("x",)),
    ("confining_flux_dropped", "q[ax] = p->D_s * s->thetac[x] * n[ax];\n        eq_scalar(s->c[x]",
     "q[ax] = 0.0 * s->thetac[x] * n[ax];\n        eq_scalar(s->c[x]",
     pins.test_reduces_to_the_2d_oracle, ("z",)),
    ("theta_factor", "s->theta[x] = (4.0 / p->W)", "s->theta[x] = (2.0 / p->W)",
     pins.test_reduces_to_the_2d_oracle, ("x",)),
    ("all_moments_relaxed_with_w", "double lam = is_first_order(k) ? w1 : 1.0;",
     "double lam = w1;", pins.test_reduces_to_the_2d_oracle, ("y",)),
    ("stream_direction_z", "k - E3[a][2]);", "k + E3[a][2]);",
     pins.test_reduces_to_the_2d_oracle, ("x",)),
    ("mobility_for_surfactant", "const double w_chi = rate_from_coeff(p->D_s);",
     "const double w_chi = rate_from_coeff(p->M_phi);",
     pins.test_sphere_surface_mode_decay, (1,)),
    # the flow lattice
    ("flow_eq_psi_sign", "m == 1 ? -u[ax] : CS2 + u[ax] * u[ax];", "m == 1 ? u[ax] : CS2 + u[ax] * u[ax];",
     fpins.test_flow_equilibrium_raw_moments, ()),
    ("trace_without_m002", "B[a][a] = 1.0;  B[a][b] = 1.0;  B[a][c] = 1.0;",
     "B[a][a] = 1.0;  B[a][b] = 1.0;  B[a][c] = 0.0;", fpins.test_sound_wave_in_three_dimensions, ()),
    ("trace_relaxed_with_nu", "if (k == 2) lam = w_zeta;", "if (k == 2) lam = w_nu;",
     fpins.test_sound_wave_in_three_dimensions, ()),
    ("first_order_source_sign", "sg[first[a]] = CS2 * Ft[a] - u[a] * G;",
     "sg[first[a]] = CS2 * Ft[a] + u[a] * G;", fpins.test_flow_reduces_to_the_2d_coupled_oracle, ("z",)),
    ("moving_wall_term", "2.0 * weight(a) * s->rho[x] * (E3[a][0] * uw)",
     "1.0 * weight(a) * s->rho[x] * (E3[a][0] * uw)", fpins.test_flow_reduces_to_the_2d_coupled_oracle, ("z",)),
    ("marangoni_projection", "(gs[ax] - n[ax] * nds)", "(gs[ax])",
     fpins.test_flow_reduces_to_the_2d_coupled_oracle, ("z",)),
    ("curvature_without_z", "acc += weight(q) * (E3[q][0] * n[0] + E3[q][1] * n[1] + E3[q][2] * n[2]);",
     "acc += weight(q) * (E3[q][0] * n[0] + E3[q][1] * n[1]);", fpins.test_curvature_of_sphere_and_cylinder, ()),
    ("half_force_in_velocity", "u[ax] = (s->jv[ax][x] + 0.5 * CS2 * s->Ft[ax][x]) / (CS2 * rho);",
     "u[ax] = (s->jv[ax][x] + 1.0 * CS2 * s->Ft[ax][x]) / (CS2 * rho);",
     fpins.test_flow_reduces_to_the_2d_coupled_oracle, ("z",)),
    ("xz_shear_at_rate_one", "if (k == 6 || k == 18 || k == 4 || k == 10 || k == 12) lam = w_nu;",
     "if (k == 6 || k == 18 || k == 4 || k == 12) lam = w_nu;",
     fpins.test_flow_reduces_to_the_2d_coupled_oracle, ("y",)),
]


@pytest.mark.parametrize("tag,old,new,pin,args", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(tmp_path, monkeypatch, tag, old, new, pin, args):
    mod = _build_variant(str(tmp_path), tag, old, new)
    with pytest.raises(AssertionError):
        _run_pin(monkeypatch, mod, pin, *args)

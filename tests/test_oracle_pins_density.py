"""Pins of the oracle's variable-density, variable-viscosity path (App. D).

Every other pin runs at rho_a = rho_b and nu_a = nu_b, where the density
interpolation, psi = P - rho cs2 and the F_p parts of the second-order
sources drop out.  These pins run at density and viscosity ratios of 2 to 5
against what the mathematics fixes:

  * equilibrium raw moments at rho != 1 (sum e g = rho cs2 u, App. D);
  * a flat interface between unequal densities at rest stays at rest with
    uniform P (exact);
  * sound in each bulk phase: speed cs, decay (nu + zeta) k^2 / 2 with that
    phase's nu, and velocity amplitude P' / (rho cs) (linear acoustics of the
    macroscopic equations of App. D);
  * a stratified layer translated parallel to its interfaces: Galilean
    invariance fixes u = U exactly; the scheme's residual must vanish at
    second order in 1/W.  Axis-aligned, only sigma_11's F_p terms act on it;
    along a diagonal, sigma_20 and sigma_02's F_p terms do;
  * two-layer Couette flow: the shear stress mu du/dy is uniform, with
    mu = rho(phi) nu(phi), so u(y) = -U + tau int_0^y dy' / mu(y').

Each pin is a function returning the measured quantity, so that
tests/test_oracle_mutations.py can run it against deliberately broken copies
of the oracle and show that it fails there.
"""
import math

import numpy as np
import pytest

from paper_2504_09024_gb300 import workloads as W

CS2 = 1.0 / 3.0
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WQ = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def rho_of_phi(phi, ra, rb, pa=1.0, pb=0.0):
    """rho = rho_b + (phi - phi_b) / (phi_a - phi_b) (rho_a - rho_b) (App. D)."""
    return rb + (phi - pb) / (pa - pb) * (ra - rb)


# ---------------------------------------------------------------------------
# Measurements (each returns numbers; the tests below hold them to bounds)
# ---------------------------------------------------------------------------

def equilibrium_moment_errors(orc, ra=2.5, rb=0.5):
    """Largest deviation of the brute-force raw moments of g^eq from
    sum g = P, sum e g = rho cs2 u, sum e_x^2 g = cs2 P + rho cs2 ux^2,
    sum e_x e_y g = rho cs2 ux uy, at several phi between the phases, and of
    the rest equilibrium from w_q P."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(4):
        phi0 = rng.uniform(0.0, 1.0)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        Pv = CS2 * rng.uniform(0.6, 1.4)
        phys = W.Physics(nx=6, ny=5, mode=0, rho_a=ra, rho_b=rb)
        s = orc.Sim(phys)
        one = np.ones((5, 6))
        s.init(phi0 * one, 0 * one, ux * one, uy * one, Pv * one)
        g = s.pops()["g"][:, 2, 3]
        rho = rho_of_phi(phi0, ra, rb)
        errs = [
            g.sum() - Pv,
            (EX * g).sum() - rho * CS2 * ux,
            (EY * g).sum() - rho * CS2 * uy,
            (EX ** 2 * g).sum() - (CS2 * Pv + rho * CS2 * ux ** 2),
            (EY ** 2 * g).sum() - (CS2 * Pv + rho * CS2 * uy ** 2),
            (EX * EY * g).sum() - rho * CS2 * ux * uy,
        ]
        worst = max(worst, max(abs(e) for e in errs))
        # at rest the equilibrium is w_q P whatever the density
        s.init(phi0 * one, 0 * one, 0 * one, 0 * one, Pv * one)
        g0 = s.pops()["g"][:, 2, 3]
        worst = max(worst, np.abs(g0 - WQ * Pv).max())
    return worst


def flat_interface_at_rest(orc, steps=400):
    """Max |u| and the spread of P after `steps` on a periodic stratified
    layer, rho_a / rho_b = 2, nu_a / nu_b = 2, at rest with uniform P."""
    nx, ny = 4, 64
    phys = W.Physics(nx=nx, ny=ny, walls_y=0, mode=0, W=4.0, M_phi=0.02, D_s=0.02,
                     nu_a=0.1, nu_b=0.05, rho_a=2.0, rho_b=1.0)
    phi, c = W.flat_band_fields(nx, ny, ny / 4, 3 * ny / 4, 4.0)
    z = np.zeros_like(phi)
    s = orc.Sim(phys)
    s.init(phi, c, z, z)
    s.step(steps)
    F = s.fields()
    return max(np.abs(F["ux"]).max(), np.abs(F["uy"]).max()), np.ptp(F["P"])


def bulk_sound(orc, phase, ra=2.5, rb=0.5, na=0.08, nb=0.02, zeta=0.05, T=300, nx=64):
    """A travelling pressure wave in a uniform phase (phi = phi_a or phi_b).
    Returns (speed / cs, decay rate / ((nu + zeta) k^2 / 2), |u'| rho cs / |P'|)."""
    eps, cs = 1e-6, math.sqrt(CS2)
    phys = W.Physics(nx=nx, ny=4, walls_y=0, mode=0, nu_a=na, nu_b=nb, zeta=zeta,
                     rho_a=ra, rho_b=rb)
    X, _ = W.cell_centres(nx, 4)
    k = 2 * np.pi / nx
    xx = X - 0.5
    rho, nu = (ra, na) if phase == "a" else (rb, nb)
    phi = np.full_like(X, 1.0 if phase == "a" else 0.0)
    P0 = CS2 * 0.5 * (ra + rb)
    s = orc.Sim(phys)
    s.init(phi, 0 * X, eps / (rho * cs) * np.cos(k * xx), 0 * X, P0 + eps * np.cos(k * xx))
    ph, amp, ratio = [], [], []
    for _ in range(T):
        F = s.fields()
        zP = 2 * ((F["P"][0] - P0) * np.exp(1j * k * xx[0])).mean()
        zu = 2 * (F["ux"][0] * np.exp(1j * k * xx[0])).mean()
        ph.append(np.angle(zP))
        amp.append(abs(zP) / eps)
        ratio.append(abs(zu) / abs(zP))
        s.step(1)
    t = np.arange(T)
    speed = np.polyfit(t, np.unwrap(ph), 1)[0] / k
    rate = -np.polyfit(t, np.log(amp), 1)[0]
    return speed / cs, rate / ((nu + zeta) * k ** 2 / 2), float(np.mean(ratio)) * rho * cs


def translated_layer(orc, Wd, diagonal=False, U=0.05, steps=None):
    """Stratified layer (rho_a / rho_b = 2, nu_a / nu_b = 2) on a periodic box,
    moving at uniform U parallel to its interfaces.  Returns max |u - U| / U
    after the run (the exact solution is u = U for all time)."""
    if diagonal:
        n = int(16 * Wd)
        nx = ny = n
    else:
        nx, ny = 4, int(16 * Wd)
    steps = steps or int((500 if diagonal else 750) * Wd)
    phys = W.Physics(nx=nx, ny=ny, walls_y=0, mode=0, W=Wd, M_phi=0.02, D_s=0.02,
                     nu_a=0.1, nu_b=0.05, rho_a=2.0, rho_b=1.0)
    X, Y = W.cell_centres(nx, ny)
    if diagonal:
        s_ = np.mod(X + Y, nx)  # interfaces along x + y = const, flow along (1, -1)
        zeta = np.minimum(s_ - nx / 4, 3 * nx / 4 - s_) / math.sqrt(2)
        ux = np.full_like(X, U / math.sqrt(2))
        uy = -ux
    else:
        zeta = np.minimum(Y - ny / 4, 3 * ny / 4 - Y)
        ux = np.full_like(X, U)
        uy = np.zeros_like(X)
    phi = 0.5 + 0.5 * np.tanh(2 * zeta / Wd)
    s = orc.Sim(phys)
    s.init(phi, 0 * phi, ux, uy)
    s.step(steps)
    F = s.fields()
    return max(np.abs(F["ux"] - ux).max(), np.abs(F["uy"] - uy).max()) / U


def two_layer_couette(orc, ny=64, Wd=4.0, U=0.01, steps=60000, ra=2.0, rb=1.0,
                      na=1 / 6, nb=1 / 12):
    """Walls at y = 0 (-U) and y = H (+U), fluid a in the middle half.
    Returns (max |u - u_exact| / U, max |u_y| / U), u_exact from the uniform
    shear stress with mu = rho(phi) nu(phi) of the run's own phase field."""
    nx = 4
    phys = W.Physics(nx=nx, ny=ny, walls_y=1, mode=0, u_wall=U, W=Wd, M_phi=0.02, D_s=0.02,
                     nu_a=na, nu_b=nb, rho_a=ra, rho_b=rb)
    phi, c = W.flat_band_fields(nx, ny, ny / 4, 3 * ny / 4, Wd)
    z = np.zeros_like(phi)
    s = orc.Sim(phys)
    s.init(phi, c, z, z)
    s.step(steps)
    F = s.fields()
    ph = F["phi"][:, 0]
    mu = rho_of_phi(ph, ra, rb) * (nb + ph * (na - nb))
    inv = 1.0 / mu
    # integral of 1/mu from the wall plane y = 0 to each cell centre (trapezoid
    # between centres, half a cell of the first value at the wall)
    cum = np.concatenate([[0.5 * inv[0]], 0.5 * inv[0] + np.cumsum(0.5 * (inv[:-1] + inv[1:]))])
    total = cum[-1] + 0.5 * inv[-1]
    u_exact = -U + (2 * U / total) * cum
    return np.abs(F["ux"][:, 0] - u_exact).max() / U, np.abs(F["uy"]).max() / U


# ---------------------------------------------------------------------------
# Bounds
# ---------------------------------------------------------------------------

EQ_TOL = 1e-15
SOUND_TOL = dict(speed=2e-3, rate=0.02, impedance=5e-3)
LAYER_W4_TOL = 0.03        # axis-aligned, W = 4 (measured 0.018)
LAYER_ORDER = (0.2, 0.35)  # residual ratio per doubling of W: second order gives 1/4
DIAG_W4_TOL = 0.03         # diagonal, W = 4 (measured 0.009)
COUETTE_TOL = 0.01         # W = 4 (measured 0.0042)


def test_flow_equilibrium_moments_unequal_densities(oracle_mod):
    assert equilibrium_moment_errors(oracle_mod) < EQ_TOL


def test_flat_interface_unequal_densities_at_rest(oracle_mod):
    umax, dP = flat_interface_at_rest(oracle_mod)
    assert umax < 1e-14 and dP < 1e-14


@pytest.mark.parametrize("phase", ["a", "b"])
def test_sound_in_each_bulk_phase(oracle_mod, phase):
    """rho_a = 2.5, rho_b = 0.5, nu_a = 0.08, nu_b = 0.02: each phase carries
    sound at cs with its own viscous decay and impedance rho cs."""
    speed, rate, imp = bulk_sound(oracle_mod, phase)
    assert abs(speed - 1) < SOUND_TOL["speed"], speed
    assert abs(rate - 1) < SOUND_TOL["rate"], rate
    assert abs(imp - 1) < SOUND_TOL["impedance"], imp


def test_translated_layer_galilean_axis_aligned(oracle_mod):
    """sigma_11 = cs2 (F_px u_y + F_py u_x) + ...: with rho varying across the
    layer and u along it, F_py u_x cancels the spurious shear stress the
    density gradient puts into the second-order moments.  The residual falls
    at second order in 1/W (W = 4, 8, 16)."""
    r = [translated_layer(oracle_mod, Wd) for Wd in (4.0, 8.0, 16.0)]
    assert r[0] < LAYER_W4_TOL, r
    for a, b in zip(r, r[1:]):
        assert LAYER_ORDER[0] < b / a < LAYER_ORDER[1], r


def test_translated_layer_galilean_diagonal(oracle_mod):
    """Along a lattice diagonal the F_px u_x and F_py u_y terms of sigma_20 and
    sigma_02 act as well."""
    r = translated_layer(oracle_mod, 4.0, diagonal=True)
    assert r < DIAG_W4_TOL, r


def test_two_layer_couette_density_and_viscosity_ratio(oracle_mod):
    """mu_a / mu_b = (2 x 1/6) / (1 x 1/12) = 4: the steady profile has slopes
    in the ratio 1/4 inside and out, joined across the diffuse interface."""
    err, uy = two_layer_couette(oracle_mod)
    assert err < COUETTE_TOL, err
    assert uy < 1e-10

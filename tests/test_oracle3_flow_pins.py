"""Pins of the 3-D (D3Q27) oracle's flow lattice: App. D carried to three
axes by the product rule (the readings are in oracle/lbm_oracle3.c).

  * the raw moments of the flow equilibria: rho cs2 times a Maxwellian's plus
    psi times the weights' (1, 0, cs2) per axis, and their fixed point;
  * exact reduction to the pinned 2-D coupled oracle for fields uniform along
    z (moving walls, tension, Marangoni stress, density ratio 2), along x
    (resting walls, body force) and along y (periodic), at nu = zeta, where
    the trace of the second-order moments relaxes like the rest and the
    reduction is exact;
  * acoustics at nu != zeta: a standing wave decays at ((4/3) nu + (2/3) zeta)
    k^2 / 2, the three-dimensional Chapman-Enskog result for a trace relaxed
    with zeta = cs2 (1/w - 1/2) (the 2-D rate (nu + zeta) k^2 / 2 is rejected);
  * Poiseuille flow between resting walls at nu != zeta;
  * the curvature div n: -2/R on a sphere, -1/R on a cylinder;
  * a spherical drop in a diagonal stream translates with it, stays
    spherical and keeps the 3-D Laplace jump 2 sigma / R.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2504_09024_gb300 import workloads as W

CS2 = 1.0 / 3.0


def _raw(pops, vel, m, n, p):
    e = vel.astype(np.float64)
    return np.tensordot(e[:, 0] ** m * e[:, 1] ** n * e[:, 2] ** p, pops, axes=(0, 0))


def test_flow_equilibrium_raw_moments():
    """Uniform phi between the phases (rho = 1.6 of rho_a = 2, rho_b = 1), a
    uniform velocity and the rest pressure P = cs2 (rho_a + rho_b) / 2: each
    raw moment of g is rho cs2 prod(1, u, cs2 + u^2) + psi prod(1, 0, cs2),
    psi = P - rho cs2, and stays so through three steps."""
    s = oracle.Sim3(4, 4, 4, W=3.0, flow=True, rho_a=2.0, rho_b=1.0, nu_a=0.1, nu_b=0.1)
    u = (0.04, -0.03, 0.02)
    phi = np.full(s.shape, 0.6)
    s.init(phi, np.zeros(s.shape), *u)
    rho = 1.0 + 0.6
    P = CS2 * 1.5
    psi = P - rho * CS2
    vel = oracle.velocities3()

    def check(g):
        for m in range(3):
            for n in range(3):
                for p in range(3):
                    maxw = 1.0
                    wts = 1.0
                    for k, ui in zip((m, n, p), u):
                        maxw *= (1.0, ui, CS2 + ui * ui)[k]
                        wts *= (1.0, 0.0, CS2)[k]
                    want = rho * CS2 * maxw + psi * wts
                    assert np.allclose(_raw(g, vel, m, n, p), want, rtol=0, atol=1e-15), (m, n, p)

    check(s.flow_pops())
    s.step(3)
    check(s.flow_pops())
    fl = s.flow_fields()
    for ax, name in enumerate(("ux", "uy", "uz")):
        assert np.abs(fl[name] - u[ax]).max() < 1e-15


def _case2d(nx, ny, walls, u_wall, fext=(0.0, 0.0)):
    nu = 0.12
    phys = W.Physics(nx=nx, ny=ny, walls_y=walls, mode=0, u_wall=u_wall, W=3.0, M_phi=0.02,
                     D_s=0.02, nu_a=nu, nu_b=nu, zeta=nu, rho_a=2.0, rho_b=1.0, sigma_o=5e-3,
                     beta=0.3, c_max=1.0, fext_x=fext[0], fext_y=fext[1])
    phi, c = W.drop_fields(nx, ny, 5.0, 3.0, xc=0.48 * nx, yc=0.51 * ny,
                           c_of_theta=lambda t: 0.3 + 0.15 * np.cos(t) + 0.05 * np.sin(2 * t))
    if walls and u_wall:
        ux, uy = W.shear_profile(nx, ny, u_wall)
    else:
        X, Y = W.cell_centres(nx, ny)
        ux = 0.01 * np.sin(2 * np.pi * Y / ny)
        uy = 0.008 * np.cos(2 * np.pi * X / nx)
    return phys, phi, c, ux, uy


def _sim3(phys, shape, fext3):
    nz, ny, nx = shape
    return oracle.Sim3(nx, ny, nz, W=phys.W, M_phi=phys.M_phi, D_s=phys.D_s, flow=True,
                       walls_y=phys.walls_y, u_wall=phys.u_wall, nu_a=phys.nu_a, nu_b=phys.nu_b,
                       zeta=phys.zeta, rho_a=phys.rho_a, rho_b=phys.rho_b,
                       sigma_o=phys.sigma_o, beta=phys.beta, c_max=phys.c_max, fext=fext3)


@pytest.mark.parametrize("uniform_axis", ["z", "x", "y"])
def test_flow_reduces_to_the_2d_coupled_oracle(uniform_axis):
    depth, steps = 2, 30
    if uniform_axis == "z":    # 2-D (x, y) -> 3-D (x, y); walls moving along x
        phys, phi2, c2, ux2, uy2 = _case2d(30, 20, 1, 0.02)
        ny2, nx2 = phi2.shape
        shape = (depth, ny2, nx2)
        expand = lambda a: np.ascontiguousarray(np.broadcast_to(a[None, :, :], shape))
        fext3 = (0.0, 0.0, 0.0)
        to3 = lambda f: (f["ux"], f["uy"], None)
    elif uniform_axis == "x":  # 2-D (x, y) -> 3-D (z, y); resting walls, body force
        phys, phi2, c2, ux2, uy2 = _case2d(24, 20, 1, 0.0, fext=(2e-5, 0.0))
        ny2, nx2 = phi2.shape
        shape = (nx2, ny2, depth)
        expand = lambda a: np.ascontiguousarray(np.broadcast_to(a.T[:, :, None], shape))
        fext3 = (0.0, 0.0, 2e-5)
        to3 = lambda f: (None, f["uy"], f["ux"])
    else:                      # 2-D (x, y) -> 3-D (x, z); periodic
        phys, phi2, c2, ux2, uy2 = _case2d(26, 22, 0, 0.0)
        ny2, nx2 = phi2.shape
        shape = (ny2, depth, nx2)
        expand = lambda a: np.ascontiguousarray(np.broadcast_to(a[:, None, :], shape))
        fext3 = (0.0, 0.0, 0.0)
        to3 = lambda f: (f["ux"], None, f["uy"])
    s2 = oracle.Sim(phys)
    s2.init(phi2, c2, ux2, uy2)
    s3 = _sim3(phys, shape, fext3)
    zero = np.zeros_like(phi2)
    u3 = [expand(v if v is not None else zero) for v in to3({"ux": ux2, "uy": uy2})]
    s3.init(expand(phi2), expand(c2), *u3)
    s2.step(steps)
    s3.step(steps)
    f2, f3, fl3 = s2.fields(), s3.fields(), s3.flow_fields()
    assert np.abs(f2["phi"] - phi2).max() > 1e-3
    for name in ("phi", "c"):
        assert np.abs(f3[name] - expand(f2[name])).max() < 1e-13, name
    assert np.abs(fl3["P"] - expand(f2["P"])).max() < 1e-13
    for comp, want in zip(("ux", "uy", "uz"), to3(f2)):
        want = np.zeros_like(phi2) if want is None else want
        assert np.abs(fl3[comp] - expand(want)).max() < 1e-13, comp


def test_sound_wave_in_three_dimensions():
    """A standing pressure wave along x oscillates at cs k and decays at
    ((4/3) nu + (2/3) zeta) k^2 / 2 (nu = 0.05, zeta = 0.2)."""
    nx, nu, zeta, eps = 64, 0.05, 0.2, 1e-6
    s = oracle.Sim3(nx, 2, 2, W=3.0, flow=True, nu_a=nu, nu_b=nu, zeta=zeta)
    X, _, _ = W.cell_centres3(nx, 2, 2)
    k = 2 * np.pi / nx
    z = np.zeros(s.shape)
    s.init(z, z, P=CS2 + eps * np.cos(k * (X - 0.5)))
    amps = []
    T = 600
    for _ in range(T):
        P = s.flow_fields()["P"]
        amps.append(2 * ((P[0, 0] - CS2) * np.cos(k * (X[0, 0] - 0.5))).mean())
        s.step(1)
    a = np.array(amps) / eps
    t = np.arange(T)
    omega = math.sqrt(CS2) * k

    def dev(gam):
        return np.abs(a - np.exp(-gam * t) * np.cos(omega * t)).max()

    assert dev(((4.0 / 3.0) * nu + (2.0 / 3.0) * zeta) * k ** 2 / 2) < 0.02
    assert dev((nu + zeta) * k ** 2 / 2) > 0.05


def test_poiseuille_between_resting_walls():
    """u(y) = F y (H - y) / (2 rho nu) at nu = 1/6, zeta = 0.05."""
    nx, ny, nz, Fx, nu = 4, 16, 2, 1e-6, 1.0 / 6.0
    s = oracle.Sim3(nx, ny, nz, W=3.0, flow=True, walls_y=1, nu_a=nu, nu_b=nu, zeta=0.05,
                    fext=(Fx, 0.0, 0.0))
    z = np.zeros(s.shape)
    s.init(z, z)
    s.step(6000)
    fl = s.flow_fields()
    _, Y, _ = W.cell_centres3(nx, ny, nz)
    exact = Fx * Y * (ny - Y) / (2 * nu)
    assert np.abs(fl["ux"] - exact).max() / exact.max() < 0.01
    assert np.abs(fl["uy"]).max() < 1e-12 and np.abs(fl["uz"]).max() < 1e-12


def test_curvature_of_sphere_and_cylinder():
    n, R, Wd = 32, 9.0, 3.0
    phi, c = W.sphere_fields(n, n, n, R, Wd)
    s = oracle.Sim3(n, n, n, W=Wd)
    s.init(phi, c)
    kap = s.curvature()
    X, Y, Z = W.cell_centres3(n, n, n)
    r = np.sqrt((X - n / 2) ** 2 + (Y - n / 2) ** 2 + (Z - n / 2) ** 2)
    band = np.abs(r - R) < 0.5
    assert abs((kap[band] * r[band]).mean() + 2.0) < 0.01
    phi2, _ = W.drop_fields(n, n, R, Wd)
    phic = np.ascontiguousarray(np.broadcast_to(phi2[None], (4, n, n)))
    s2 = oracle.Sim3(n, n, 4, W=Wd)
    s2.init(phic, np.zeros_like(phic))
    kap2 = s2.curvature()[0]
    X2, Y2 = W.cell_centres(n, n)
    r2 = np.hypot(X2 - n / 2, Y2 - n / 2)
    b2 = np.abs(r2 - R) < 0.5
    assert abs((kap2[b2] * r2[b2]).mean() + 1.0) < 0.01


def test_translating_sphere():
    """A clean spherical drop in a uniform diagonal stream (all three axes
    active) translates with it, stays spherical and keeps the 3-D Laplace
    jump 2 sigma / R (times the discrete tension factor of the profile)."""
    from test_oracle_pins import _discrete_tension_factor
    n, R, Wd, sig, T = 20, 5.0, 3.0, 1e-3, 200
    U = (0.02, 0.015, -0.01)
    phi, c = W.sphere_fields(n, n, n, R, Wd)
    s = oracle.Sim3(n, n, n, W=Wd, M_phi=0.05, D_s=0.1, flow=True, nu_a=1.0 / 6.0,
                    nu_b=1.0 / 6.0, zeta=0.5, sigma_o=sig)
    s.init(phi, c, *U, P=CS2 + 2 * sig / R * phi)
    X, Y, Z = W.cell_centres3(n, n, n)

    def centroid(ph):
        w = np.clip(ph, 0, 1)
        out = []
        for A in (X, Y, Z):
            ang = 2 * np.pi * A / n
            out.append((np.arctan2((w * np.sin(ang)).sum(), (w * np.cos(ang)).sum()) * n
                        / (2 * np.pi)) % n)
        return np.array(out)

    c0 = centroid(s.fields()["phi"])
    s.step(T)
    ph = s.fields()["phi"]
    c1 = centroid(ph)
    moved = (c1 - c0 + n / 2) % n - n / 2
    assert np.abs(moved - np.array(U) * T).max() < 1e-3 * 0.02 * T
    d = [((A - cc + n / 2) % n) - n / 2 for A, cc in zip((X, Y, Z), c1)]
    w = np.clip(ph, 0, 1)
    M = np.array([[(w * d[i] * d[j]).sum() for j in range(3)] for i in range(3)]) / w.sum()
    ev = np.linalg.eigvalsh(M)
    assert (ev.max() - ev.min()) / ev.mean() < 1e-4
    r = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
    P = s.flow_fields()["P"]
    dP = P[r < R - 3].mean() - P[r > R + 4].mean()
    assert abs(dP * R / (2 * sig * _discrete_tension_factor(Wd)) - 1) < 0.06

"""Pins of the 3-D (D3Q27) oracle of the two scalar lattices.

Each test fixes the oracle against something other than itself:
  * the raw moments of its discrete equilibria against those of a Maxwellian
    (every one of the 27, at a non-zero velocity);
  * its gradient stencil against the closed form of the stencil applied to a
    product of sines (which fixes the rest, face, edge and corner weights);
  * the exact reduction to the pinned 2-D oracle for fields uniform along one
    axis, for each of the three axes (the z-marginal of a D3Q27 run of a
    z-uniform field is a D2Q9 run);
  * the decay of the surface modes l = 1 and l = 2 of the surfactant on a
    sphere, whose rate l (l + 1) D_s / R^2 is the closed form of surface
    diffusion on a sphere (3-D form of the static drop of Sec. 4.1);
  * conservation of sum phi and sum c under a non-uniform velocity.
"""
import numpy as np
import pytest

import oracle
from paper_2504_09024_gb300 import workloads as wl

CS2 = 1.0 / 3.0


def _raw_moment(pops, vel, m, n, p):
    e = vel.astype(np.float64)
    w = (e[:, 0] ** m) * (e[:, 1] ** n) * (e[:, 2] ** p)
    return np.tensordot(w, pops, axes=(0, 0))


def test_equilibrium_raw_moments_are_maxwellian():
    """Uniform fields (no interface, so no flux): each raw moment of the
    initial populations is prod_i r(m_i, u_i), r(0) = 1, r(1) = u,
    r(2) = cs2 + u^2 -- the moments of a Maxwellian, times the density --
    and stays so through three steps."""
    n = 4
    s = oracle.Sim3(n, n, n, W=3.0)
    u = (0.07, -0.045, 0.031)
    phi = np.full(s.shape, 0.37)
    c = np.full(s.shape, 0.21)
    s.init(phi, c, *u)
    pops = s.pops()
    vel = oracle.velocities3()
    assert len({tuple(v) for v in vel}) == 27 and np.abs(vel).max() == 1

    def r(k, ui):
        return (1.0, ui, CS2 + ui * ui)[k]

    def check(pops):
        for m in range(3):
            for nn in range(3):
                for p in range(3):
                    want = r(m, u[0]) * r(nn, u[1]) * r(p, u[2])
                    for name, dens in (("f", 0.37), ("h", 0.21)):
                        got = _raw_moment(pops[name], vel, m, nn, p)
                        assert np.allclose(got, dens * want, rtol=0, atol=1e-15), (name, m, nn, p)

    check(pops)
    # the uniform equilibrium is a fixed point of collision and streaming
    s.step(3)
    check(s.pops())


def test_gradient_of_product_of_sines():
    """d_x of sin(kx) sin(ly) sin(mz) through the stencil is
    sin(k) cos(kx) (2/3 + cos(l)/3) sin(ly) (2/3 + cos(m)/3) sin(mz), and
    likewise on the other axes: the closed form of the D3Q27 weights."""
    nx, ny, nz = 10, 8, 12
    s = oracle.Sim3(nx, ny, nz, W=3.0)
    X, Y, Z = wl.cell_centres3(nx, ny, nz)
    k, l, m = 2 * np.pi / nx, 2 * np.pi * 2 / ny, 2 * np.pi / nz
    a = np.sin(k * X) * np.sin(l * Y) * np.sin(m * Z)
    gx, gy, gz = s.gradient(a)

    def side(t):
        return 2.0 / 3.0 + np.cos(t) / 3.0

    ex = np.sin(k) * np.cos(k * X) * side(l) * np.sin(l * Y) * side(m) * np.sin(m * Z)
    ey = side(k) * np.sin(k * X) * np.sin(l) * np.cos(l * Y) * side(m) * np.sin(m * Z)
    ez = side(k) * np.sin(k * X) * side(l) * np.sin(l * Y) * np.sin(m) * np.cos(m * Z)
    for got, want in ((gx, ex), (gy, ey), (gz, ez)):
        assert np.abs(got - want).max() < 1e-13


def _case2d(nx=18, ny=14):
    phys = wl.Physics(nx=nx, ny=ny, walls_y=0, mode=1, W=3.0, M_phi=0.07, D_s=0.09)
    phi, c = wl.drop_fields(nx, ny, 4.5, 3.0, xc=8.3, yc=7.1,
                            c_of_theta=lambda t: 0.4 + 0.2 * np.cos(t) + 0.1 * np.sin(2 * t))
    X, Y = wl.cell_centres(nx, ny)
    ux = 0.03 * np.sin(2 * np.pi * Y / ny) + 0.01
    uy = 0.02 * np.cos(2 * np.pi * X / nx) - 0.015
    return phys, phi, c, ux, uy


@pytest.mark.parametrize("uniform_axis", ["z", "x", "y"])
def test_reduces_to_the_2d_oracle(uniform_axis):
    """A field uniform along one axis evolves as the 2-D oracle evolves its
    cross-section: the 3-D phi and c equal the 2-D ones to rounding."""
    phys, phi2, c2, ux2, uy2 = _case2d()
    ny2, nx2 = phi2.shape
    depth = 3
    zero = np.zeros_like(phi2)
    if uniform_axis == "z":      # 2-D (x, y) -> 3-D (x, y)
        shape, expand = (depth, ny2, nx2), (lambda a: np.broadcast_to(a[None, :, :], (depth, ny2, nx2)))
        u = (ux2, uy2, zero)
    elif uniform_axis == "x":    # 2-D (x, y) -> 3-D (y, z)
        shape, expand = (ny2, nx2, depth), (lambda a: np.broadcast_to(a[:, :, None], (ny2, nx2, depth)))
        u = (zero, ux2, uy2)
    else:                        # 2-D (x, y) -> 3-D (x, z)
        shape, expand = (ny2, depth, nx2), (lambda a: np.broadcast_to(a[:, None, :], (ny2, depth, nx2)))
        u = (ux2, zero, uy2)
    nz3, ny3, nx3 = shape
    s3 = oracle.Sim3(nx3, ny3, nz3, W=phys.W, M_phi=phys.M_phi, D_s=phys.D_s)
    s3.init(expand(phi2), expand(c2), *[expand(v) for v in u])
    s2 = oracle.Sim(phys)
    s2.init(phi2, c2, ux2, uy2)
    steps = 40
    s2.step(steps)
    s3.step(steps)
    f2, f3 = s2.fields(), s3.fields()
    assert np.abs(f2["phi"] - phi2).max() > 1e-3      # the case moves
    for name in ("phi", "c"):
        assert np.abs(f3[name] - expand(f2[name])).max() < 1e-13, name


@pytest.mark.parametrize("mode", [1, 2])
def test_sphere_surface_mode_decay(mode):
    """Surface diffusion on a sphere: the mode P_l(mu) of c decays at
    l (l + 1) D_s / R^2 (2 for l = 1, 6 for l = 2; a 2-D circle gives l^2)."""
    n, R, W, D = 24, 7.0, 3.0, 0.1
    case = wl.sphere_surface_mode(n=n, R=R, W=W, D_s=D, M_phi=0.05, mode=mode)
    s = oracle.Sim3(n, n, n, W=W, M_phi=case.M_phi, D_s=D)
    s.init(case.phi, case.c)
    X, Y, Z = wl.cell_centres3(n, n, n)
    dx, dy, dz = X - n / 2, Y - n / 2, Z - n / 2
    mu = dz / np.sqrt(dx * dx + dy * dy + dz * dz)
    Pl = mu if mode == 1 else 0.5 * (3 * mu * mu - 1)

    def amp():
        return float((s.fields()["c"] * Pl).sum())

    a0 = amp()
    s.step(case.steps)
    rate = -np.log(amp() / a0) / case.steps
    ratio = rate / (mode * (mode + 1) * D / R ** 2)
    assert 0.92 < ratio < 1.03, ratio


def test_conservation_under_a_nonuniform_velocity():
    n = 12
    s = oracle.Sim3(n, n + 2, n - 2, W=3.0, M_phi=0.05, D_s=0.08)
    phi, c = wl.sphere_fields(n, n + 2, n - 2, 3.5, 3.0, c_of_cos=lambda m: 0.3 + 0.1 * m)
    X, Y, Z = wl.cell_centres3(n, n + 2, n - 2)
    ux = 0.03 * np.sin(2 * np.pi * Z / (n - 2))
    uy = 0.02 * np.cos(2 * np.pi * X / n)
    uz = 0.025 * np.sin(2 * np.pi * Y / (n + 2))
    s.init(phi, c, ux, uy, uz)
    s0 = s.fields()
    s.step(60)
    s1 = s.fields()
    assert np.abs(s1["phi"] - s0["phi"]).max() > 1e-3
    for name in ("phi", "c"):
        assert abs(s1[name].sum() - s0[name].sum()) < 1e-11 * abs(s0[name].sum())


def test_far_field_surfactant_is_set_by_the_rounding_of_phi():
    """Where |grad phi| is at the rounding level of phi (far from the drop)
    the normal, and the confining flux that moves the little surfactant
    there, follow the smallest changes of phi.  A random perturbation of phi
    of 3e-7 -- the size of an FP32-arithmetic path's own phi error -- moves
    the far-field c by a sizeable part of its value, while c where the normal
    is defined (|grad phi| > 1e-5) moves by about the perturbation, relative.
    This is what makes the far-field c not unique at FP32 precision."""
    n = 32
    case = wl.sphere_surface_mode(n=n, R=8.0, W=3.0, D_s=0.1, M_phi=0.05, mode=1,
                                  u=(0.02, -0.013, 0.009), steps=200)
    pert = 3e-7 * np.random.default_rng(5).standard_normal(case.phi.shape)
    out = []
    for phi in (case.phi, case.phi + pert):
        s = oracle.Sim3(n, n, n, W=case.W, M_phi=case.M_phi, D_s=case.D_s)
        s.init(phi, case.c, *case.u)
        s.step(case.steps)
        f = s.fields()
        g = s.gradient(f["phi"])
        out.append((f["c"], np.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)))
    (ca, ga), (cb, _) = out
    m = ga > 1e-5
    dc = cb - ca
    assert np.linalg.norm(dc[m]) < 1e-6 * np.linalg.norm(ca[m])
    assert np.abs(dc[~m]).max() > 0.1 * np.abs(ca[~m]).max()

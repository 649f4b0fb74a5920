"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the only code shared by the CUDA path and the FP64 oracle.
It builds initial macroscopic fields and physical parameter sets; it holds
none of the lattice Boltzmann arithmetic (no populations, moments,
equilibria, relaxation rates or stencils).

Sources for the shapes:
  * interface profile  phi = phi_m + phi_o tanh(2 zeta / W)        (Sec. 2.2, Eq. CACEeq)
  * surfactant profile c = c_hat(theta) / cosh^2(2 zeta / W)       (Sec. 2.2, Eq. ISSeq; Sec. 4.1)
  * zeta = R - |x - x_o| for a circular drop                         (Sec. 4.1)
  * shear start profile u(y) = U_o (2 y / H - 1)                     (Sec. 4.3)
  * Re = gamma_dot R^2 / nu, Ca = mu gamma_dot R / sigma_o,
    gamma_dot = 2 U_o / H, Pe = Re nu / D_s, Pe* = U_o W / M_phi = 0.5 (Sec. 4.3)

Coordinates: cell (i, j) has centre (i + 1/2, j + 1/2); with walls the
channel spans y in [0, ny] so the wall planes sit half a cell outside the
first and last rows.  Arrays are row-major [ny][nx], x fastest, float64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

CASE_SEED = 20250409  # fixed seed for the random ensembles (uneven-grid batches)


@dataclasses.dataclass
class Physics:
    """Physical (lattice-unit) parameters of one run.

    Transport coefficients are given directly (not as relaxation times); the
    library and the oracle each convert them to collision rates themselves.
    """
    nx: int
    ny: int
    walls_y: int = 0            # 0: periodic in y; 1: moving walls at y = 0 (-u_wall) and y = ny (+u_wall)
    mode: int = 0               # 0: coupled f + h + g; 1: prescribed velocity, f + h only
    u_wall: float = 0.0
    W: float = 4.0
    phi_a: float = 1.0
    phi_b: float = 0.0
    M_phi: float = 0.1          # CACE mobility
    D_s: float = 0.1            # surface diffusivity of the interface-bound scalar
    nu_a: float = 0.1
    nu_b: float = 0.1
    zeta: float = 1.0 / 6.0     # bulk viscosity; 1/6 is a bulk relaxation rate of 1
    rho_a: float = 1.0
    rho_b: float = 1.0
    sigma_o: float = 0.0
    beta: float = 0.0
    c_max: float = 1.0
    fext_x: float = 0.0
    fext_y: float = 0.0
    sigma_literal: int = 0      # 1: surface-tension force exactly as printed (no width normalisation)

    def as_dict(self) -> dict:
        return dataclasses.asdict(self)


@dataclasses.dataclass
class Case:
    """A run: physics plus initial macroscopic fields and a step count."""
    name: str
    phys: Physics
    phi: np.ndarray
    c: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    P: Optional[np.ndarray]
    steps: int
    meta: dict = dataclasses.field(default_factory=dict)


def cell_centres(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y, indexing="xy")  # shapes [ny][nx]


def drop_fields(nx, ny, R, W, xc=None, yc=None, phi_a=1.0, phi_b=0.0,
                c_of_theta=None, c0=0.0):
    """Circular drop: tanh phase profile and sech^2 surfactant band.

    c_of_theta(theta) gives c_hat along the interface (theta = atan2 about the
    centre); if None, c_hat = c0 uniformly.
    """
    if xc is None:
        xc = nx / 2.0
    if yc is None:
        yc = ny / 2.0
    X, Y = cell_centres(nx, ny)
    dx, dy = X - xc, Y - yc
    r = np.hypot(dx, dy)
    zeta = R - r
    phi_m = 0.5 * (phi_a + phi_b)
    phi_o = 0.5 * (phi_a - phi_b)
    phi = phi_m + phi_o * np.tanh(2.0 * zeta / W)
    theta = np.arctan2(dy, dx)
    chat = c_of_theta(theta) if c_of_theta is not None else np.full_like(r, c0)
    c = chat / np.cosh(np.clip(2.0 * zeta / W, -300.0, 300.0)) ** 2
    return phi, c


def flat_band_fields(nx, ny, y1, y2, W, phi_a=1.0, phi_b=0.0, c0=0.0):
    """A periodic slab phi_a between y1 < y < y2 with two flat interfaces."""
    X, Y = cell_centres(nx, ny)
    zeta = np.minimum(Y - y1, y2 - Y)
    phi_m = 0.5 * (phi_a + phi_b)
    phi_o = 0.5 * (phi_a - phi_b)
    phi = phi_m + phi_o * np.tanh(2.0 * zeta / W)
    c = c0 / np.cosh(np.clip(2.0 * zeta / W, -300.0, 300.0)) ** 2
    return phi, c


def shear_profile(nx, ny, u_wall):
    """u(y) = U_o (2 y / H - 1) with H = ny and y the cell-centre height."""
    _, Y = cell_centres(nx, ny)
    ux = u_wall * (2.0 * Y / ny - 1.0)
    return ux, np.zeros_like(ux)


@dataclasses.dataclass
class ShearDerived:
    gamma_dot: float
    U_o: float
    sigma_o: float
    D_s: float
    M_phi: float


def shear_drop_parameters(H, R, W, nu, rho, Re, Ca, Pe_s, Pe_star=0.5) -> ShearDerived:
    """Drop-in-shear parameter set from the dimensionless groups of Sec. 4.3.

    Re = gamma_dot R^2 / nu, gamma_dot = 2 U_o / H, Ca = rho nu gamma_dot R / sigma_o,
    Pe_s = Re nu / D_s, Pe* = U_o W / M_phi.
    """
    gamma_dot = Re * nu / R ** 2
    U_o = gamma_dot * H / 2.0
    sigma_o = rho * nu * gamma_dot * R / Ca
    D_s = Re * nu / Pe_s
    M_phi = U_o * W / Pe_star
    return ShearDerived(gamma_dot, U_o, sigma_o, D_s, M_phi)


# ---------------------------------------------------------------------------
# The five workload shapes.
# ---------------------------------------------------------------------------

def static_drop_cos_mode(nx=128, ny=128, R=32.0, W=4.0, D_s=0.1, M_phi=0.1,
                         steps=2000, amp=0.1, base=0.5) -> Case:
    """Plain method, small: f + h lattices, u = 0, periodic box, stationary
    drop with c_hat = base + amp cos(theta) on the interface (Sec. 4.1 shape)."""
    phys = Physics(nx=nx, ny=ny, walls_y=0, mode=1, W=W, M_phi=M_phi, D_s=D_s)
    phi, c = drop_fields(nx, ny, R, W, c_of_theta=lambda t: base + amp * np.cos(t))
    z = np.zeros_like(phi)
    return Case("static_drop_cos_mode", phys, phi, c, z, z.copy(), None, steps,
                meta=dict(R=R, amp=amp, base=base))


def shear_drop(nx, ny, R, W, Ca, beta, Gamma0, Re=0.1, Pe_s=10.0, nu=0.1,
               rho=1.0, c_max=1.0, steps=1000, name="shear_drop") -> Case:
    """Insoluble-surfactant drop in simple shear between moving walls
    (Sec. 4.3 set-up), density and viscosity ratio 1."""
    d = shear_drop_parameters(ny, R, W, nu, rho, Re, Ca, Pe_s)
    phys = Physics(nx=nx, ny=ny, walls_y=1, mode=0, u_wall=d.U_o, W=W,
                   M_phi=d.M_phi, D_s=d.D_s, nu_a=nu, nu_b=nu,
                   rho_a=rho, rho_b=rho, sigma_o=d.sigma_o, beta=beta,
                   c_max=c_max)
    phi, c = drop_fields(nx, ny, R, W, c0=Gamma0)
    ux, uy = shear_profile(nx, ny, d.U_o)
    return Case(name, phys, phi, c, ux, uy, None, steps,
                meta=dict(R=R, Ca=Ca, beta=beta, Gamma0=Gamma0, Re=Re,
                          Pe_s=Pe_s, gamma_dot=d.gamma_dot))


def shear_drop_512x256(steps=40000) -> Case:
    """Full coupled 3-lattice workload: 512x256, R = 48, W = 4, Ca = 0.2,
    Re = 0.1, beta = 0.2, Gamma0 = 0.3, Pe_s = 10, nu = 0.1."""
    return shear_drop(512, 256, 48.0, 4.0, Ca=0.2, beta=0.2, Gamma0=0.3,
                      steps=steps, name="shear_drop_512x256")


def shear_drop_2048x1024(Ca=0.1, steps=5000) -> Case:
    """Precision / bandwidth workload: 2048x1024, R = 192, W = 5, beta = 0.3,
    Gamma0 = 0.3, Re = 0.1, Pe_s = 10, Ca in {0.1, 0.3}."""
    return shear_drop(2048, 1024, 192.0, 5.0, Ca=Ca, beta=0.3, Gamma0=0.3,
                      steps=steps, name=f"shear_drop_2048x1024_Ca{Ca:g}")


ENSEMBLE_GRIDS = ((256, 128), (512, 256), (768, 384), (1024, 512))


def ensemble_draws(nruns=64, seed=CASE_SEED, grids=ENSEMBLE_GRIDS):
    """Random drop-in-shear ensemble: grid ~ U{grids}, R = H/5,
    Ca ~ U[0.05, 0.5], beta ~ U[0, 0.5], Pe_s ~ logU[1, 100],
    Gamma0 ~ U[0.1, 0.6].  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nruns):
        nx, ny = grids[int(rng.integers(len(grids)))]
        out.append(dict(nx=nx, ny=ny, R=ny / 5.0,
                        Ca=float(rng.uniform(0.05, 0.5)),
                        beta=float(rng.uniform(0.0, 0.5)),
                        Pe_s=float(math.exp(rng.uniform(math.log(1.0), math.log(100.0)))),
                        Gamma0=float(rng.uniform(0.1, 0.6))))
    return out


def ensemble_case(draw, shrink=1, W=4.0, steps=20000) -> Case:
    """Drop-in-shear case of one ensemble draw; `shrink` divides the grid (and
    so R = H/5) for test-sized versions of the same ensemble."""
    nx, ny = draw["nx"] // shrink, draw["ny"] // shrink
    return shear_drop(nx, ny, ny / 5.0, W, Ca=draw["Ca"], beta=draw["beta"],
                      Gamma0=draw["Gamma0"], Pe_s=draw["Pe_s"], steps=steps,
                      name=f"ensemble_{nx}x{ny}")


def lively_shear_drop(nx=100, ny=60, R=14.0, W=4.0, steps=400) -> Case:
    """A small, fast-evolving drop in shear used for parity tests: strong
    shear, tension and Marangoni stress so that every term moves within a few
    hundred steps; the grid is ragged with respect to the kernels' tiles."""
    U = 0.02
    phys = Physics(nx=nx, ny=ny, walls_y=1, mode=0, u_wall=U, W=W,
                   M_phi=0.02, D_s=0.02, nu_a=0.1, nu_b=0.1,
                   rho_a=1.0, rho_b=1.0, sigma_o=5e-3, beta=0.3, c_max=1.0)
    phi, c = drop_fields(nx, ny, R, W,
                         c_of_theta=lambda t: 0.3 + 0.15 * np.cos(t) + 0.05 * np.sin(2 * t))
    ux, uy = shear_profile(nx, ny, U)
    return Case("lively_shear_drop", phys, phi, c, ux, uy, None, steps)


# ---- three-dimensional workloads (D3Q27 scalar lattices, prescribed u) -----

@dataclasses.dataclass
class Case3:
    """A 3-D run of the two scalar lattices under a prescribed velocity.

    Fields are [nz][ny][nx] float64 (x fastest), periodic on every axis; the
    velocity is either three constants or three fields of that shape.
    """
    name: str
    nx: int
    ny: int
    nz: int
    W: float
    M_phi: float
    D_s: float
    phi: np.ndarray
    c: np.ndarray
    u: tuple
    steps: int
    phi_a: float = 1.0
    phi_b: float = 0.0
    meta: dict = dataclasses.field(default_factory=dict)


def cell_centres3(nx: int, ny: int, nz: int):
    """Cell centres (i + 1/2, j + 1/2, k + 1/2) as three [nz][ny][nx] arrays."""
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5,
                          indexing="ij")
    return x, y, z


def sphere_fields(nx, ny, nz, R, W, centre=None, phi_a=1.0, phi_b=0.0,
                  c_of_cos=None, c0=0.0):
    """Spherical drop: tanh phase profile and sech^2 surfactant band.

    c_of_cos(mu) gives c_hat on the interface as a function of the polar
    cosine mu = (z - z_o) / |x - x_o| (axis along z); if None, c_hat = c0.
    """
    if centre is None:
        centre = (nx / 2.0, ny / 2.0, nz / 2.0)
    X, Y, Z = cell_centres3(nx, ny, nz)
    dx, dy, dz = X - centre[0], Y - centre[1], Z - centre[2]
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    zeta = R - r
    phi_m = 0.5 * (phi_a + phi_b)
    phi_o = 0.5 * (phi_a - phi_b)
    phi = phi_m + phi_o * np.tanh(2.0 * zeta / W)
    mu = np.where(r > 0.0, dz / np.maximum(r, 1e-300), 0.0)
    chat = c_of_cos(mu) if c_of_cos is not None else np.full_like(r, c0)
    c = chat / np.cosh(np.clip(2.0 * zeta / W, -300.0, 300.0)) ** 2
    return phi, c


def sphere_surface_mode(n=256, R=None, W=4.0, D_s=0.1, M_phi=0.1, mode=1, amp=0.1,
                        base=0.5, u=(0.0, 0.0, 0.0), steps=None) -> Case3:
    """A spherical drop of radius R in an n^3 periodic box carrying the surface
    mode c_hat = base + amp P_l(mu) (l = 1 or 2) of its surfactant: the 3-D
    form of the static drop of Sec. 4.1; with u != 0 the drop is advected as in
    the second case of Sec. 4.1.  The default length is one e-folding time of
    the mode, R^2 / (l (l + 1) D_s)."""
    if R is None:
        R = n / 4.0
    legendre = {1: lambda m: m, 2: lambda m: 0.5 * (3.0 * m * m - 1.0)}[mode]
    phi, c = sphere_fields(n, n, n, R, W, c_of_cos=lambda m: base + amp * legendre(m))
    if steps is None:
        steps = int(round(R * R / (mode * (mode + 1) * D_s)))
    return Case3(f"sphere_{n}^3_l{mode}", n, n, n, W, M_phi, D_s, phi, c, tuple(u), steps,
                 meta=dict(R=R, mode=mode, amp=amp, base=base))

"""FP64 CPU oracle of the coupled central-moment LBM (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
may import this package.  The product path (``paper_2504_09024_gb300``) never
imports it and shares no code with it.

The C source ``lbm_oracle.c`` computes each collision with the literal 9x9
matrices of the paper (P and P^-1 of App. A; F(u), F^-1(u) generated from the
binomial definition, Eq. cmscalar; B and B^-1 of App. D) in the order of the
algorithm lists of Sec. 3, App. C and App. D.  ``mlp.py`` holds the FP64
reference of the surrogate network.

Parity status of each function is recorded in the repository's design notes;
the pins live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liblbm_oracle.so")
_SRC = [os.path.join(_HERE, "lbm_oracle.c"), os.path.join(_HERE, "lbm_oracle3.c")]
_HDRS = [os.path.join(_HERE, "lbm_oracle.h"), os.path.join(_HERE, "lbm_oracle3.h")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle with gcc into oracle/_lib/liblbm_oracle.so."""
    os.makedirs(_LIBDIR, exist_ok=True)
    # the build flags live in this file: a change to it rebuilds too
    newest = max(os.path.getmtime(p) for p in _SRC + _HDRS + [os.path.abspath(__file__)])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
    cmds = [base[:1] + ["-fopenmp"] + base[1:]] if openmp else []
    cmds.append(base)
    err = None
    for cmd in cmds:
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, _SO)
            return _SO
        err = r.stderr
    raise RuntimeError(f"oracle build failed:\n{err}")


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("walls_y", ctypes.c_int),
        ("mode", ctypes.c_int), ("sigma_literal", ctypes.c_int), ("pad_", ctypes.c_int),
        ("u_wall", ctypes.c_double), ("W", ctypes.c_double), ("phi_a", ctypes.c_double),
        ("phi_b", ctypes.c_double), ("M_phi", ctypes.c_double), ("D_s", ctypes.c_double),
        ("nu_a", ctypes.c_double), ("nu_b", ctypes.c_double), ("zeta", ctypes.c_double),
        ("rho_a", ctypes.c_double), ("rho_b", ctypes.c_double), ("sigma_o", ctypes.c_double),
        ("beta", ctypes.c_double), ("c_max", ctypes.c_double), ("fext_x", ctypes.c_double),
        ("fext_y", ctypes.c_double),
    ]


class OrcDiag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_longlong), ("sum_phi", ctypes.c_double), ("sum_c", ctypes.c_double),
        ("D", ctypes.c_double), ("L", ctypes.c_double), ("B", ctypes.c_double),
        ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("umax", ctypes.c_double),
        ("nonfinite", ctypes.c_longlong), ("sigma_neg", ctypes.c_longlong),
    ]


class Orc3Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("pad_", ctypes.c_int),
        ("W", ctypes.c_double), ("phi_a", ctypes.c_double), ("phi_b", ctypes.c_double),
        ("M_phi", ctypes.c_double), ("D_s", ctypes.c_double),
        ("mode", ctypes.c_int), ("walls_y", ctypes.c_int), ("sigma_literal", ctypes.c_int),
        ("pad2_", ctypes.c_int),
        ("u_wall", ctypes.c_double), ("nu_a", ctypes.c_double), ("nu_b", ctypes.c_double),
        ("zeta", ctypes.c_double), ("rho_a", ctypes.c_double), ("rho_b", ctypes.c_double),
        ("sigma_o", ctypes.c_double), ("beta", ctypes.c_double), ("c_max", ctypes.c_double),
        ("fext", ctypes.c_double * 3),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_create.restype = ctypes.c_void_p
            L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_init.argtypes = [ctypes.c_void_p] + [_DP] * 5
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_get_step.restype = ctypes.c_longlong
            L.orc_get_step.argtypes = [ctypes.c_void_p]
            L.orc_fields.argtypes = [ctypes.c_void_p] + [_DP] * 5
            L.orc_geometry.argtypes = [ctypes.c_void_p] + [_DP] * 6
            L.orc_get_pops.argtypes = [ctypes.c_void_p] + [_DP] * 3
            L.orc_set_pops.argtypes = [ctypes.c_void_p] + [_DP] * 3
            L.orc_set_velocity.argtypes = [ctypes.c_void_p] + [_DP] * 2
            L.orc_reset_f.argtypes = [ctypes.c_void_p, _DP]
            L.orc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.POINTER(OrcDiag)]
            L.orc_matrix_P.argtypes = [_DP]
            L.orc_matrix_Pinv.argtypes = [_DP]
            L.orc_matrix_F.argtypes = [ctypes.c_double, ctypes.c_double, _DP]
            L.orc_matrix_Finv.argtypes = [ctypes.c_double, ctypes.c_double, _DP]
            L.orc_gradient.argtypes = [ctypes.c_void_p, _DP, _DP, _DP]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc3_create.restype = ctypes.c_void_p
            L.orc3_create.argtypes = [ctypes.POINTER(Orc3Params)]
            L.orc3_destroy.argtypes = [ctypes.c_void_p]
            L.orc3_init.argtypes = [ctypes.c_void_p] + [_DP] * 5
            L.orc3_init_pressure.argtypes = [ctypes.c_void_p] + [_DP] * 6
            L.orc3_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc3_get_step.restype = ctypes.c_longlong
            L.orc3_get_step.argtypes = [ctypes.c_void_p]
            L.orc3_fields.argtypes = [ctypes.c_void_p, _DP, _DP]
            L.orc3_normals.argtypes = [ctypes.c_void_p] + [_DP] * 3
            L.orc3_get_pops.argtypes = [ctypes.c_void_p, _DP, _DP]
            L.orc3_set_pops.argtypes = [ctypes.c_void_p, _DP, _DP]
            L.orc3_velocities.argtypes = [ctypes.POINTER(ctypes.c_int)]
            for name in ("orc3_matrix_P", "orc3_matrix_Pinv"):
                getattr(L, name).argtypes = [_DP]
            for name in ("orc3_matrix_F", "orc3_matrix_Finv"):
                getattr(L, name).argtypes = [ctypes.c_double] * 3 + [_DP]
            L.orc3_gradient.argtypes = [ctypes.c_void_p] + [_DP] * 4
            L.orc3_flow_fields.argtypes = [ctypes.c_void_p] + [_DP] * 4
            L.orc3_get_flow_pops.argtypes = [ctypes.c_void_p, _DP]
            L.orc3_curvature.argtypes = [ctypes.c_void_p, _DP]
            _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _arr(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def params_from(phys) -> OrcParams:
    d = phys.as_dict() if hasattr(phys, "as_dict") else dict(phys)
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        if name in d:
            setattr(p, name, d[name])
    return p


def matrix(name, ux=0.0, uy=0.0):
    out = np.zeros(81)
    L = lib()
    if name == "P":
        L.orc_matrix_P(_ptr(out))
    elif name == "Pinv":
        L.orc_matrix_Pinv(_ptr(out))
    elif name == "F":
        L.orc_matrix_F(ux, uy, _ptr(out))
    elif name == "Finv":
        L.orc_matrix_Finv(ux, uy, _ptr(out))
    else:
        raise ValueError(name)
    return out.reshape(9, 9)


def num_threads() -> int:
    return lib().orc_num_threads()


class Sim:
    """One oracle run.  Fields are [ny][nx] float64; populations [9][ny][nx]."""

    def __init__(self, phys):
        self.phys = phys
        self.nx, self.ny = int(phys.nx), int(phys.ny)
        self._p = params_from(phys)
        self._h = lib().orc_create(ctypes.byref(self._p))
        if not self._h:
            raise ValueError("oracle: invalid parameters")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi, c, ux, uy, P=None):
        a = [_arr(v) for v in (phi, c, ux, uy, P)]
        lib().orc_init(self._h, *[_ptr(v) for v in a])

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    @property
    def t(self):
        return lib().orc_get_step(self._h)

    def fields(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(5)]
        lib().orc_fields(self._h, *[_ptr(v) for v in out])
        return dict(zip(("phi", "c", "ux", "uy", "P"), out))

    def geometry(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(6)]
        lib().orc_geometry(self._h, *[_ptr(v) for v in out])
        return dict(zip(("nx", "ny", "gmag", "kappa", "Fsx", "Fsy"), out))

    def pops(self):
        out = [np.zeros((9, self.ny, self.nx)) for _ in range(3)]
        lib().orc_get_pops(self._h, *[_ptr(v) for v in out])
        return dict(zip(("f", "h", "g"), out))

    def set_pops(self, f=None, h=None, g=None):
        a = [_arr(v) for v in (f, h, g)]
        lib().orc_set_pops(self._h, *[_ptr(v) for v in a])

    def set_velocity(self, ux, uy):
        a = [_arr(v) for v in (ux, uy)]
        lib().orc_set_velocity(self._h, *[_ptr(v) for v in a])

    def reset_f(self, phi):
        a = _arr(phi)
        lib().orc_reset_f(self._h, _ptr(a))

    def gradient(self, field):
        a = _arr(field)
        gx = np.zeros_like(a)
        gy = np.zeros_like(a)
        lib().orc_gradient(self._h, _ptr(a), _ptr(gx), _ptr(gy))
        return gx, gy

    def diagnostics(self):
        d = OrcDiag()
        lib().orc_diagnostics(self._h, ctypes.byref(d))
        return {name: getattr(d, name) for name, _ in OrcDiag._fields_}


def run_case(case, steps=None):
    """Convenience: build, initialise and advance an oracle run of a workload Case."""
    s = Sim(case.phys)
    s.init(case.phi, case.c, case.ux, case.uy, case.P)
    s.step(case.steps if steps is None else steps)
    return s


# ---- D3Q27 scalar lattices under a prescribed velocity (lbm_oracle3.c) -----

def matrix3(name, ux=0.0, uy=0.0, uz=0.0):
    """The 27 x 27 matrices P, P^-1, F(u), F^-1(u) of the 3-D oracle."""
    out = np.zeros(729)
    L = lib()
    if name in ("P", "Pinv"):
        getattr(L, f"orc3_matrix_{name}")(_ptr(out))
    elif name in ("F", "Finv"):
        getattr(L, f"orc3_matrix_{name}")(ux, uy, uz, _ptr(out))
    else:
        raise ValueError(name)
    return out.reshape(27, 27)


def velocities3():
    """The 27 velocities of the 3-D oracle in its population order, [27][3]."""
    buf = (ctypes.c_int * 81)()
    lib().orc3_velocities(buf)
    return np.array(list(buf), dtype=np.int64).reshape(27, 3)


class Sim3:
    """One 3-D oracle run.  Fields are [nz][ny][nx] float64, periodic in x and
    z, and in y unless walls_y.  flow=True couples the D3Q27 flow lattice
    (the remaining keywords are its physics, as for the 2-D oracle)."""

    def __init__(self, nx, ny, nz, W=4.0, phi_a=1.0, phi_b=0.0, M_phi=0.1, D_s=0.1,
                 flow=False, walls_y=0, u_wall=0.0, nu_a=0.1, nu_b=0.1, zeta=1.0 / 6.0,
                 rho_a=1.0, rho_b=1.0, sigma_o=0.0, beta=0.0, c_max=1.0, fext=(0.0, 0.0, 0.0),
                 sigma_literal=0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self._p = Orc3Params(nx=self.nx, ny=self.ny, nz=self.nz, W=W, phi_a=phi_a,
                             phi_b=phi_b, M_phi=M_phi, D_s=D_s, mode=1 if flow else 0,
                             walls_y=int(walls_y), sigma_literal=int(sigma_literal),
                             u_wall=u_wall, nu_a=nu_a, nu_b=nu_b, zeta=zeta, rho_a=rho_a,
                             rho_b=rho_b, sigma_o=sigma_o, beta=beta, c_max=c_max)
        for i in range(3):
            self._p.fext[i] = float(fext[i])
        self._h = lib().orc3_create(ctypes.byref(self._p))
        if not self._h:
            raise ValueError("oracle: invalid 3-D parameters")

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if self._h:
            lib().orc3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi, c, ux=0.0, uy=0.0, uz=0.0, P=None):
        u = [np.broadcast_to(np.asarray(v, dtype=np.float64), self.shape) for v in (ux, uy, uz)]
        a = [_arr(v) for v in (phi, c, *u)]
        if P is None:
            lib().orc3_init(self._h, *[_ptr(v) for v in a])
        else:
            Pa = _arr(np.broadcast_to(np.asarray(P, dtype=np.float64), self.shape))
            lib().orc3_init_pressure(self._h, *[_ptr(v) for v in a], _ptr(Pa))

    def step(self, n=1):
        lib().orc3_step(self._h, int(n))

    @property
    def t(self):
        return lib().orc3_get_step(self._h)

    def fields(self):
        phi, c = np.zeros(self.shape), np.zeros(self.shape)
        lib().orc3_fields(self._h, _ptr(phi), _ptr(c))
        return {"phi": phi, "c": c}

    def normals(self):
        out = [np.zeros(self.shape) for _ in range(3)]
        lib().orc3_normals(self._h, *[_ptr(v) for v in out])
        return out

    def pops(self):
        f, h = np.zeros((27,) + self.shape), np.zeros((27,) + self.shape)
        lib().orc3_get_pops(self._h, _ptr(f), _ptr(h))
        return {"f": f, "h": h}

    def flow_fields(self):
        out = [np.zeros(self.shape) for _ in range(4)]
        lib().orc3_flow_fields(self._h, *[_ptr(v) for v in out])
        return dict(zip(("ux", "uy", "uz", "P"), out))

    def curvature(self):
        k = np.zeros(self.shape)
        lib().orc3_curvature(self._h, _ptr(k))
        return k

    def flow_pops(self):
        g = np.zeros((27,) + self.shape)
        lib().orc3_get_flow_pops(self._h, _ptr(g))
        return g

    def set_pops(self, f=None, h=None):
        a = [_arr(v) for v in (f, h)]
        lib().orc3_set_pops(self._h, *[_ptr(v) for v in a])

    def gradient(self, field):
        a = _arr(field)
        g = [np.zeros_like(a) for _ in range(3)]
        lib().orc3_gradient(self._h, _ptr(a), *[_ptr(v) for v in g])
        return g

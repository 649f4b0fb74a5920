"""Thin ctypes binding of the 3-D scalar lattices in liblbm.so (include/lbm3.h).

Functions carry the C names and only marshal arguments; every step runs in
the library's CUDA kernels, and there is no CPU fallback.  Field arrays are
float64 [nz][ny][nx]; population arrays float64 [27][nz][ny][nx] in the
order of ``lbm3_velocities()``.  Host arguments are C-contiguous float64
numpy arrays; ``*_device`` functions take CUDA torch tensors or raw device
addresses.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Optional

import numpy as np

from . import lbm as _lbm
from .lbm import LBM_OK, LBMError, _addr

LBM3_MAX_CELLS = 1 << 30


class lbm3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("velocity_field", ctypes.c_int32),
        ("W", ctypes.c_double), ("phi_a", ctypes.c_double), ("phi_b", ctypes.c_double),
        ("M_phi", ctypes.c_double), ("D_s", ctypes.c_double), ("u", ctypes.c_double * 3),
    ]


_VP = ctypes.c_void_p
_DP = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)

# Every symbol include/lbm3.h declares, with (restype, argtypes).
SIGNATURES3 = {
    "lbm3_params_default": (ctypes.c_int, [ctypes.POINTER(lbm3_params)]),
    "lbm3_create": (ctypes.c_int, [ctypes.POINTER(lbm3_params), _VP, ctypes.POINTER(_VP)]),
    "lbm3_destroy": (None, [_VP]),
    "lbm3_init_fields": (ctypes.c_int, [_VP] + [_DP] * 5),
    "lbm3_init_fields_device": (ctypes.c_int, [_VP] + [_DP] * 5),
    "lbm3_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "lbm3_get_fields": (ctypes.c_int, [_VP, _DP, _DP]),
    "lbm3_get_fields_device": (ctypes.c_int, [_VP, _DP, _DP]),
    "lbm3_get_populations": (ctypes.c_int, [_VP, _DP, _DP]),
    "lbm3_get_populations_device": (ctypes.c_int, [_VP, _DP, _DP]),
    "lbm3_sums": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double)]),
    "lbm3_velocities": (ctypes.c_int, [_I32P]),
    "lbm3_synchronize": (ctypes.c_int, [_VP]),
    "lbm3_get_step": (ctypes.c_int64, [_VP]),
    "lbm3_set_launch_shape": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "lbm3_get_launch_shape": (ctypes.c_int, [_VP, _I32P, _I32P]),
    "lbm3_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, _I32P, _I32P,
                                     ctypes.POINTER(ctypes.c_double)]),
}

_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """The library with the lbm3_* signatures set."""
    global _lib
    with _lock:
        if _lib is None:
            L = _lbm.load(build_if_missing)
            for name, (res, args) in SIGNATURES3.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(code, where):
    if code != LBM_OK:
        raise LBMError(code, where)
    return code


def lbm3_params_default() -> lbm3_params:
    p = lbm3_params()
    _check(load().lbm3_params_default(ctypes.byref(p)), "lbm3_params_default")
    return p


def lbm3_create(p: lbm3_params, stream: Optional[int] = None) -> int:
    h = _VP()
    _check(load().lbm3_create(ctypes.byref(p), stream, ctypes.byref(h)), "lbm3_create")
    return h.value


def lbm3_destroy(ctx: int) -> None:
    load().lbm3_destroy(ctx)


def lbm3_init_fields(ctx, phi, c, ux=None, uy=None, uz=None):
    args = [_addr(v) for v in (phi, c, ux, uy, uz)]
    _check(load().lbm3_init_fields(ctx, *args), "lbm3_init_fields")


def lbm3_init_fields_device(ctx, phi, c, ux=None, uy=None, uz=None):
    args = [_addr(v) for v in (phi, c, ux, uy, uz)]
    _check(load().lbm3_init_fields_device(ctx, *args), "lbm3_init_fields_device")


def lbm3_step(ctx, nsteps: int):
    _check(load().lbm3_step(ctx, int(nsteps)), "lbm3_step")


def lbm3_get_fields(ctx, phi=None, c=None):
    _check(load().lbm3_get_fields(ctx, _addr(phi), _addr(c)), "lbm3_get_fields")


def lbm3_get_fields_device(ctx, phi=None, c=None):
    _check(load().lbm3_get_fields_device(ctx, _addr(phi), _addr(c)), "lbm3_get_fields_device")


def lbm3_get_populations(ctx, f=None, h=None):
    _check(load().lbm3_get_populations(ctx, _addr(f), _addr(h)), "lbm3_get_populations")


def lbm3_get_populations_device(ctx, f=None, h=None):
    _check(load().lbm3_get_populations_device(ctx, _addr(f), _addr(h)),
           "lbm3_get_populations_device")


def lbm3_sums(ctx):
    out = (ctypes.c_double * 3)()
    _check(load().lbm3_sums(ctx, out), "lbm3_sums")
    return {"sum_phi": out[0], "sum_c": out[1], "nonfinite": int(out[2])}


def lbm3_velocities() -> np.ndarray:
    buf = (ctypes.c_int32 * 81)()
    _check(load().lbm3_velocities(buf), "lbm3_velocities")
    return np.array(list(buf), dtype=np.int64).reshape(27, 3)


def lbm3_synchronize(ctx):
    _check(load().lbm3_synchronize(ctx), "lbm3_synchronize")


def lbm3_get_step(ctx) -> int:
    return int(load().lbm3_get_step(ctx))


def lbm3_set_launch_shape(ctx, rows=0, seg_z=0):
    _check(load().lbm3_set_launch_shape(ctx, int(rows), int(seg_z)), "lbm3_set_launch_shape")


def lbm3_get_launch_shape(ctx):
    r, s = ctypes.c_int32(), ctypes.c_int32()
    _check(load().lbm3_get_launch_shape(ctx, ctypes.byref(r), ctypes.byref(s)),
           "lbm3_get_launch_shape")
    return r.value, s.value


def lbm3_autotune(ctx, steps=4):
    r, s, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().lbm3_autotune(ctx, int(steps), ctypes.byref(r), ctypes.byref(s), ctypes.byref(ms)),
           "lbm3_autotune")
    return r.value, s.value, ms.value


class Sim3:
    """One 3-D run on the GPU (a Case3 from workloads, or explicit sizes)."""

    def __init__(self, nx, ny, nz, W=4.0, phi_a=1.0, phi_b=0.0, M_phi=0.1, D_s=0.1,
                 u=(0.0, 0.0, 0.0), velocity_field=False, stream=None):
        p = lbm3_params_default()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.W, p.phi_a, p.phi_b, p.M_phi, p.D_s = W, phi_a, phi_b, M_phi, D_s
        p.velocity_field = 1 if velocity_field else 0
        for i in range(3):
            p.u[i] = float(u[i])
        self.nx, self.ny, self.nz = p.nx, p.ny, p.nz
        self.ctx = lbm3_create(p, stream)

    @classmethod
    def from_case(cls, case, stream=None):
        field = any(np.ndim(v) > 0 for v in case.u)
        u = (0.0, 0.0, 0.0) if field else tuple(float(v) for v in case.u)
        s = cls(case.nx, case.ny, case.nz, W=case.W, phi_a=case.phi_a, phi_b=case.phi_b,
                M_phi=case.M_phi, D_s=case.D_s, u=u, velocity_field=field, stream=stream)
        s.init(case.phi, case.c, *(case.u if field else (None, None, None)))
        return s

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "ctx", None):
            lbm3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi, c, ux=None, uy=None, uz=None):
        arrs = [None if v is None else np.ascontiguousarray(np.broadcast_to(v, self.shape),
                                                            dtype=np.float64)
                for v in (phi, c, ux, uy, uz)]
        lbm3_init_fields(self.ctx, *arrs)

    def step(self, n=1):
        lbm3_step(self.ctx, n)

    @property
    def t(self):
        return lbm3_get_step(self.ctx)

    def fields(self):
        phi, c = np.zeros(self.shape), np.zeros(self.shape)
        lbm3_get_fields(self.ctx, phi, c)
        return {"phi": phi, "c": c}

    def pops(self):
        f, h = np.zeros((27,) + self.shape), np.zeros((27,) + self.shape)
        lbm3_get_populations(self.ctx, f, h)
        return {"f": f, "h": h}

    def sums(self):
        return lbm3_sums(self.ctx)

    def synchronize(self):
        lbm3_synchronize(self.ctx)

"""Thin ctypes binding of liblbm.so (include/lbm.h).

Functions carry the C names and only marshal arguments: every step of the
method runs in the library's CUDA kernels.  There is no CPU fallback; if the
library is missing or fails to load, the first call raises.

Field arrays are float64 [ny][nx]; population arrays float64 [9][ny][nx].
Host arguments may be numpy arrays (any float64 C-contiguous buffer) or
pinned torch CPU tensors; ``*_device`` functions take CUDA torch tensors (or
raw integer device pointers).
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_ERR_INVALID_ARG = -1
LBM_ERR_RATE = -2
LBM_ERR_SIGMA_NEG = -3
LBM_ERR_CUDA = -4
LBM_ERR_NONFINITE = -5
LBM_ERR_TIMEOUT = -6
LBM_ERR_UNSUPPORTED = -7
LBM_ERR_IO = -8
LBM_ERR_NOMEM = -9

LBM_F32, LBM_F16S, LBM_BF16S = 1, 2, 3
LBM_COUPLED, LBM_FIXED_U = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_SPLIT, LBM_KERNEL_FUSED, LBM_KERNEL_TMA = 0, 1, 2, 3


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("walls_y", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("dtype", ctypes.c_int32), ("kernel", ctypes.c_int32),
        ("sigma_literal", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("u_wall", ctypes.c_double), ("W", ctypes.c_double), ("phi_a", ctypes.c_double),
        ("phi_b", ctypes.c_double), ("M_phi", ctypes.c_double), ("D_s", ctypes.c_double),
        ("nu_a", ctypes.c_double), ("nu_b", ctypes.c_double), ("zeta", ctypes.c_double),
        ("rho_a", ctypes.c_double), ("rho_b", ctypes.c_double), ("sigma_o", ctypes.c_double),
        ("beta", ctypes.c_double), ("c_max", ctypes.c_double), ("fext_x", ctypes.c_double),
        ("fext_y", ctypes.c_double),
    ]


class lbm_diag(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("sum_phi", ctypes.c_double), ("sum_c", ctypes.c_double),
        ("D", ctypes.c_double), ("L", ctypes.c_double), ("B", ctypes.c_double),
        ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("umax", ctypes.c_double),
        ("nonfinite", ctypes.c_int64), ("sigma_neg", ctypes.c_int64),
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


# Every symbol include/lbm.h declares, with (restype, argtypes).
_VP = ctypes.c_void_p
_DP = ctypes.c_void_p  # double* passed as an address
SIGNATURES = {
    "lbm_params_default": (ctypes.c_int, [ctypes.POINTER(lbm_params)]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), _VP, ctypes.POINTER(_VP)]),
    "lbm_destroy": (None, [_VP]),
    "lbm_init_fields": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP, _DP]),
    "lbm_init_fields_device": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP, _DP]),
    "lbm_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "lbm_get_fields": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP, _DP]),
    "lbm_get_fields_device": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP, _DP]),
    "lbm_get_populations": (ctypes.c_int, [_VP, _DP, _DP, _DP]),
    "lbm_set_populations": (ctypes.c_int, [_VP, _DP, _DP, _DP]),
    "lbm_diagnostics": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_diag)]),
    "lbm_synchronize": (ctypes.c_int, [_VP]),
    "lbm_get_step": (ctypes.c_int64, [_VP]),
    "lbm_kernel_in_use": (ctypes.c_int, [_VP]),
    "lbm_launches_per_step": (ctypes.c_int, [_VP]),
    "lbm_set_launch_shape": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "lbm_get_launch_shape": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "lbm_set_cells_per_thread": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_get_cells_per_thread": (ctypes.c_int32, [_VP]),
    "lbm_set_store_mode": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_get_store_mode": (ctypes.c_int32, [_VP]),
    "lbm_save_state": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "lbm_load_state": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "lbm_debug_stall_next_step": (ctypes.c_int, [_VP]),
    "lbm_field_stats_noalloc": (ctypes.c_int, [_DP, _DP, _DP, _DP, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _DP, _VP]),
    "lbm_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.POINTER(lbm_params), ctypes.c_int32, _VP,
                                        ctypes.POINTER(_VP)]),
    "lbm_batch_destroy": (None, [_VP]),
    "lbm_batch_size": (ctypes.c_int32, [_VP]),
    "lbm_batch_run": (_VP, [_VP, ctypes.c_int32]),
    "lbm_batch_step": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "lbm_batch_synchronize": (ctypes.c_int, [_VP]),
    "lbm_batch_set_form": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_batch_get_form": (ctypes.c_int32, [_VP]),
    "lbm_batch_set_launch_shape": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32]),
    "lbm_batch_set_cells_per_thread": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_batch_set_store_mode": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lbm_batch_get_launch_shape": (ctypes.c_int, [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "lbm_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_double)]),
    "lbm_count_components": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "surr_param_count": (ctypes.c_int32, []),
    "surr_create": (ctypes.c_int, [ctypes.c_uint64, _VP, ctypes.POINTER(_VP)]),
    "surr_destroy": (None, [_VP]),
    "surr_set_params": (ctypes.c_int, [_VP, _DP]),
    "surr_get_params": (ctypes.c_int, [_VP, _DP]),
    "surr_predict": (ctypes.c_int, [_VP, _DP, ctypes.c_int32, _DP, _DP]),
    "surr_grad": (ctypes.c_int, [_VP, _DP, _DP, _DP, ctypes.c_int32, _DP,
                                 ctypes.POINTER(ctypes.c_double)]),
    "surr_train": (ctypes.c_int, [_VP, _DP, _DP, _DP, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
}

LBM_FIELD_STATS_LEN = 13

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load liblbm.so (building it first if allowed and missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.SO
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"liblbm.so not built ({path}); run __graft_entry__.build()")
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = load().lbm_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where):
    if code != LBM_OK:
        raise LBMError(code, where)
    return code


def _addr(a, dtype=np.float64):
    """Address of a host or device buffer (numpy array, torch tensor, int or None)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data


# --- C-named wrappers ------------------------------------------------------

def lbm_params_default() -> lbm_params:
    p = lbm_params()
    _check(load().lbm_params_default(ctypes.byref(p)), "lbm_params_default")
    return p


def lbm_create(p: lbm_params, stream: Optional[int] = None) -> int:
    h = _VP()
    _check(load().lbm_create(ctypes.byref(p), stream, ctypes.byref(h)), "lbm_create")
    return h.value


def lbm_destroy(ctx: int) -> None:
    load().lbm_destroy(ctx)


def lbm_init_fields(ctx, phi, c, ux, uy, P=None):
    _check(load().lbm_init_fields(ctx, _addr(phi), _addr(c), _addr(ux), _addr(uy), _addr(P)),
           "lbm_init_fields")


def lbm_init_fields_device(ctx, phi, c, ux, uy, P=None):
    _check(load().lbm_init_fields_device(ctx, _addr(phi), _addr(c), _addr(ux), _addr(uy),
                                         _addr(P)), "lbm_init_fields_device")


def lbm_step(ctx, nsteps: int):
    _check(load().lbm_step(ctx, int(nsteps)), "lbm_step")


def lbm_get_fields(ctx, phi=None, c=None, ux=None, uy=None, P=None):
    _check(load().lbm_get_fields(ctx, _addr(phi), _addr(c), _addr(ux), _addr(uy), _addr(P)),
           "lbm_get_fields")


def lbm_get_fields_device(ctx, phi=None, c=None, ux=None, uy=None, P=None):
    _check(load().lbm_get_fields_device(ctx, _addr(phi), _addr(c), _addr(ux), _addr(uy),
                                        _addr(P)), "lbm_get_fields_device")


def lbm_get_populations(ctx, f=None, h=None, g=None):
    _check(load().lbm_get_populations(ctx, _addr(f), _addr(h), _addr(g)), "lbm_get_populations")


def lbm_set_populations(ctx, f=None, h=None, g=None):
    _check(load().lbm_set_populations(ctx, _addr(f), _addr(h), _addr(g)), "lbm_set_populations")


def lbm_diagnostics(ctx) -> dict:
    d = lbm_diag()
    _check(load().lbm_diagnostics(ctx, ctypes.byref(d)), "lbm_diagnostics")
    return {name: getattr(d, name) for name, _ in lbm_diag._fields_ if name != "reserved"}


def lbm_synchronize(ctx):
    _check(load().lbm_synchronize(ctx), "lbm_synchronize")


def lbm_get_step(ctx) -> int:
    return int(load().lbm_get_step(ctx))


def lbm_kernel_in_use(ctx) -> int:
    return int(load().lbm_kernel_in_use(ctx))


def lbm_launches_per_step(ctx) -> int:
    return int(load().lbm_launches_per_step(ctx))


def lbm_set_launch_shape(ctx, tile_x=0, seg_y=0):
    _check(load().lbm_set_launch_shape(ctx, int(tile_x), int(seg_y)), "lbm_set_launch_shape")


def lbm_get_launch_shape(ctx):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(load().lbm_get_launch_shape(ctx, ctypes.byref(a), ctypes.byref(b)),
           "lbm_get_launch_shape")
    return a.value, b.value


def lbm_set_cells_per_thread(ctx, cells: int):
    _check(load().lbm_set_cells_per_thread(ctx, int(cells)), "lbm_set_cells_per_thread")


def lbm_get_cells_per_thread(ctx) -> int:
    n = load().lbm_get_cells_per_thread(ctx)
    if n < 0:
        raise LBMError(n, "lbm_get_cells_per_thread")
    return n


LBM_STORE_DIRECT = 0
LBM_STORE_STAGED = 1


def lbm_set_store_mode(ctx, mode: int):
    _check(load().lbm_set_store_mode(ctx, int(mode)), "lbm_set_store_mode")


def lbm_get_store_mode(ctx) -> int:
    n = load().lbm_get_store_mode(ctx)
    if n < 0:
        raise LBMError(n, "lbm_get_store_mode")
    return n


def lbm_save_state(ctx, path: str):
    _check(load().lbm_save_state(ctx, path.encode()), "lbm_save_state")


def lbm_load_state(ctx, path: str):
    _check(load().lbm_load_state(ctx, path.encode()), "lbm_load_state")


def lbm_debug_stall_next_step(ctx):
    _check(load().lbm_debug_stall_next_step(ctx), "lbm_debug_stall_next_step")


def lbm_field_stats_noalloc(phi, c, ux, uy, nx, ny, walls_y, beta, c_max, result, stream=None,
                            phi_a=1.0, phi_b=0.0):
    """FP64 field statistics of device fields into the device array `result`
    (LBM_FIELD_STATS_LEN doubles) without any device allocation; phi_a and
    phi_b are the bulk phases of the drop indicator."""
    _check(load().lbm_field_stats_noalloc(_addr(phi), _addr(c), _addr(ux), _addr(uy), int(nx),
                                          int(ny), int(walls_y), float(beta), float(c_max),
                                          float(phi_a), float(phi_b), _addr(result), stream),
           "lbm_field_stats_noalloc")


def lbm_autotune(ctx, steps=32):
    """Returns (tile_x, seg_y, ms_per_step) of the fastest launch shape (now set)."""
    tx, sy, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().lbm_autotune(ctx, int(steps), ctypes.byref(tx), ctypes.byref(sy),
                               ctypes.byref(ms)), "lbm_autotune")
    return tx.value, sy.value, ms.value


def lbm_batch_create(params, stream: Optional[int] = None) -> int:
    arr = (lbm_params * len(params))(*params)
    out = _VP()
    _check(load().lbm_batch_create(arr, len(params), stream, ctypes.byref(out)), "lbm_batch_create")
    return out.value


def lbm_batch_destroy(b) -> None:
    load().lbm_batch_destroy(b)


def lbm_batch_size(b) -> int:
    n = load().lbm_batch_size(b)
    if n < 0:
        raise LBMError(n, "lbm_batch_size")
    return n


def lbm_batch_run(b, run: int) -> int:
    ctx = load().lbm_batch_run(b, int(run))
    if not ctx:
        raise LBMError(LBM_ERR_INVALID_ARG, "lbm_batch_run")
    return ctx


def lbm_batch_step(b, nsteps: int):
    _check(load().lbm_batch_step(b, int(nsteps)), "lbm_batch_step")


def lbm_batch_synchronize(b):
    _check(load().lbm_batch_synchronize(b), "lbm_batch_synchronize")


LBM_BATCH_CHAINS = 0
LBM_BATCH_PERSISTENT = 1


def lbm_batch_set_form(b, form: int):
    _check(load().lbm_batch_set_form(b, int(form)), "lbm_batch_set_form")


def lbm_batch_get_form(b) -> int:
    n = load().lbm_batch_get_form(b)
    if n < 0:
        raise LBMError(n, "lbm_batch_get_form")
    return n


def lbm_batch_set_store_mode(b, mode: int):
    _check(load().lbm_batch_set_store_mode(b, int(mode)), "lbm_batch_set_store_mode")


def lbm_batch_set_cells_per_thread(b, cells: int):
    _check(load().lbm_batch_set_cells_per_thread(b, int(cells)), "lbm_batch_set_cells_per_thread")


def lbm_batch_set_launch_shape(b, tile_x=0, seg_y=0):
    _check(load().lbm_batch_set_launch_shape(b, int(tile_x), int(seg_y)),
           "lbm_batch_set_launch_shape")


def lbm_batch_get_launch_shape(b):
    """Returns (tile_x, seg_y, blocks, tiles)."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(load().lbm_batch_get_launch_shape(b, *[ctypes.byref(x) for x in v]),
           "lbm_batch_get_launch_shape")
    return tuple(x.value for x in v)


def lbm_batch_autotune(b, steps=16):
    """Returns (tile_x, seg_y, ms_per_step) of the fastest batched launch shape (now set)."""
    tx, sy, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    _check(load().lbm_batch_autotune(b, int(steps), ctypes.byref(tx), ctypes.byref(sy),
                                     ctypes.byref(ms)), "lbm_batch_autotune")
    return tx.value, sy.value, ms.value


def lbm_count_components(ctx, level=0.5) -> int:
    n = ctypes.c_int32()
    _check(load().lbm_count_components(ctx, float(level), ctypes.byref(n)), "lbm_count_components")
    return n.value


def lbm_strerror(code: int) -> str:
    return load().lbm_strerror(code).decode()


# --- convenience object ----------------------------------------------------

def params_from(phys, dtype=LBM_F32, kernel=LBM_KERNEL_AUTO) -> lbm_params:
    """lbm_params from a workloads.Physics (or any object/dict with the fields)."""
    d = phys.as_dict() if hasattr(phys, "as_dict") else dict(phys)
    p = lbm_params_default()
    for name, _ in lbm_params._fields_:
        if name in d:
            setattr(p, name, d[name])
    p.dtype = dtype
    p.kernel = kernel
    return p


class Sim:
    """A context plus numpy-facing helpers (all work runs in liblbm.so)."""

    def __init__(self, phys, dtype=LBM_F32, kernel=LBM_KERNEL_AUTO, stream=None, ctx=None):
        self.nx, self.ny = int(phys.nx), int(phys.ny)
        self.mode = int(getattr(phys, "mode", 0))
        self.params = params_from(phys, dtype, kernel)
        # a context handed in (a run of a batch) belongs to its owner
        self._owned = ctx is None
        self.ctx = lbm_create(self.params, stream) if ctx is None else ctx

    def close(self):
        if getattr(self, "ctx", None):
            if self._owned:
                lbm_destroy(self.ctx)
            self.ctx = None

    def autotune(self, steps=32):
        return lbm_autotune(self.ctx, steps)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, phi, c, ux, uy, P=None):
        a = [None if v is None else np.ascontiguousarray(v, dtype=np.float64)
             for v in (phi, c, ux, uy, P)]
        lbm_init_fields(self.ctx, *a)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def sync(self):
        lbm_synchronize(self.ctx)

    @property
    def t(self):
        return lbm_get_step(self.ctx)

    def fields(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(5)]
        lbm_get_fields(self.ctx, *out)
        return dict(zip(("phi", "c", "ux", "uy", "P"), out))

    def pops(self):
        n = 2 if self.mode == LBM_FIXED_U else 3
        out = [np.zeros((9, self.ny, self.nx)) for _ in range(n)]
        lbm_get_populations(self.ctx, *out)
        return dict(zip(("f", "h", "g"), out))

    def set_pops(self, f=None, h=None, g=None):
        a = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in (f, h, g)]
        lbm_set_populations(self.ctx, *a)

    def diagnostics(self):
        return lbm_diagnostics(self.ctx)

    @property
    def kernel(self):
        return lbm_kernel_in_use(self.ctx)

    def set_launch_shape(self, tile_x=0, seg_y=0):
        lbm_set_launch_shape(self.ctx, tile_x, seg_y)

    def set_cells_per_thread(self, cells):
        lbm_set_cells_per_thread(self.ctx, cells)

    @property
    def cells_per_thread(self):
        return lbm_get_cells_per_thread(self.ctx)

    def set_store_mode(self, mode):
        lbm_set_store_mode(self.ctx, mode)

    @property
    def store_mode(self):
        return lbm_get_store_mode(self.ctx)

    def components(self, level=0.5):
        return lbm_count_components(self.ctx, level)

    def save(self, path):
        lbm_save_state(self.ctx, path)

    def load(self, path):
        lbm_load_state(self.ctx, path)


class Batch:
    """Runs advanced together by the batched kernel; ``runs[k]`` is a Sim view
    of run k (owned by the batch) for initialisation, fields and diagnostics."""

    def __init__(self, physics, dtype=LBM_F32, stream=None):
        self.params = [params_from(ph, dtype, LBM_KERNEL_TMA) for ph in physics]
        self.handle = lbm_batch_create(self.params, stream)
        self.runs = [Sim(ph, dtype, LBM_KERNEL_TMA, ctx=lbm_batch_run(self.handle, k))
                     for k, ph in enumerate(physics)]

    def close(self):
        if getattr(self, "handle", None):
            for r in self.runs:
                r.close()
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.runs)

    def step(self, n=1):
        lbm_batch_step(self.handle, n)

    def sync(self):
        lbm_batch_synchronize(self.handle)

    def set_launch_shape(self, tile_x=0, seg_y=0):
        lbm_batch_set_launch_shape(self.handle, tile_x, seg_y)

    def launch_shape(self):
        return lbm_batch_get_launch_shape(self.handle)

    def set_cells_per_thread(self, cells):
        lbm_batch_set_cells_per_thread(self.handle, cells)

    def set_store_mode(self, mode):
        lbm_batch_set_store_mode(self.handle, mode)

    @property
    def form(self):
        return lbm_batch_get_form(self.handle)

    def set_form(self, form):
        lbm_batch_set_form(self.handle, form)

    def autotune(self, steps=16):
        return lbm_batch_autotune(self.handle, steps)


# --- surrogate network -------------------------------------------------------

SURR_WIDTHS = (5, 128, 128, 128, 128, 2)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


class Surrogate:
    """The surrogate network of liblbm.so (all arithmetic in its kernels).
    Parameters travel as a list of (W [fout, fin], b [fout]) float32 pairs."""

    def __init__(self, seed=0, stream=None):
        out = _VP()
        _check(load().surr_create(int(seed), stream, ctypes.byref(out)), "surr_create")
        self.h = out.value
        self.count = int(load().surr_param_count())

    def close(self):
        if getattr(self, "h", None):
            load().surr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def flatten(params):
        return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(),
                                               np.asarray(b, np.float32).ravel()])
                               for W, b in params])

    @staticmethod
    def unflatten(flat):
        out, o = [], 0
        for fin, fout in zip(SURR_WIDTHS[:-1], SURR_WIDTHS[1:]):
            W = flat[o:o + fout * fin].reshape(fout, fin)
            o += fout * fin
            b = flat[o:o + fout]
            o += fout
            out.append([W.copy(), b.copy()])
        return out

    def set_params(self, params):
        flat = _f32(self.flatten(params))
        assert flat.size == self.count
        _check(load().surr_set_params(self.h, flat.ctypes.data), "surr_set_params")

    def get_params(self):
        flat = np.empty(self.count, np.float32)
        _check(load().surr_get_params(self.h, flat.ctypes.data), "surr_get_params")
        return self.unflatten(flat)

    def predict(self, X):
        X = _f32(X)
        n = X.shape[0]
        D = np.empty(n, np.float32)
        z = np.empty(n, np.float32)
        _check(load().surr_predict(self.h, X.ctypes.data, n, D.ctypes.data, z.ctypes.data),
               "surr_predict")
        return D, z

    def grad(self, X, yD, yB):
        X, yD, yB = _f32(X), _f32(yD), _f32(yB)
        g = np.empty(self.count, np.float32)
        loss = ctypes.c_double()
        _check(load().surr_grad(self.h, X.ctypes.data, yD.ctypes.data, yB.ctypes.data,
                                X.shape[0], g.ctypes.data, ctypes.byref(loss)), "surr_grad")
        return self.unflatten(g), loss.value

    def train(self, X, yD, yB, epochs, lr):
        X, yD, yB = _f32(X), _f32(yD), _f32(yB)
        loss = ctypes.c_double()
        _check(load().surr_train(self.h, X.ctypes.data, yD.ctypes.data, yB.ctypes.data,
                                 X.shape[0], int(epochs), float(lr), ctypes.byref(loss)),
               "surr_train")
        return loss.value

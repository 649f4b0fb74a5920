"""CPU checks of the 3-D C ABI (include/lbm3.h): every declared symbol is
exported and bound, the parameter struct has the header's layout, the
velocity order is the documented one, and parameter validation answers
before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2504_09024_gb300 import build as B
from paper_2504_09024_gb300 import lbm, lbm3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm3.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm3.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm3_[a-z_]+)\s*\(", text)))


def test_header_functions_exported(lib):
    names = declared_functions()
    assert len(names) == 17
    out = subprocess.run(["nm", "-D", "--defined-only", B.SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm3_\w+)", out))
    assert [n for n in names if n not in exported] == []
    assert sorted(lbm3.SIGNATURES3) == names


def test_struct_layout_matches_header(lib):
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "lbm3.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(lbm3_params), offsetof(lbm3_params, W),
         offsetof(lbm3_params, D_s), offsetof(lbm3_params, u));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    P = lbm3.lbm3_params
    assert vals == [ctypes.sizeof(P), P.W.offset, P.D_s.offset, P.u.offset]


def test_velocity_order(lib):
    v = lbm3.lbm3_velocities()
    E = [0, 1, -1]
    for a in range(27):
        assert tuple(v[a]) == (E[a % 3], E[(a // 3) % 3], E[a // 9])
    assert len({tuple(r) for r in v}) == 27


def _params(**kw):
    p = lbm3.lbm3_params_default()
    p.nx, p.ny, p.nz = 8, 8, 8
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,code", [
    (dict(nx=0), lbm.LBM_ERR_INVALID_ARG),
    (dict(nz=-3), lbm.LBM_ERR_INVALID_ARG),
    (dict(nx=1 << 11, ny=1 << 10, nz=1 << 10), lbm.LBM_ERR_INVALID_ARG),
    (dict(W=0.0), lbm.LBM_ERR_INVALID_ARG),
    (dict(phi_a=0.0, phi_b=0.0), lbm.LBM_ERR_INVALID_ARG),
    (dict(velocity_field=2), lbm.LBM_ERR_INVALID_ARG),
    (dict(M_phi=0.0), lbm.LBM_ERR_RATE),
    (dict(D_s=-0.1), lbm.LBM_ERR_RATE),
    (dict(W=float("nan")), lbm.LBM_ERR_INVALID_ARG),
    (dict(phi_a=2.5), lbm.LBM_ERR_INVALID_ARG),
    (dict(nx=16384, ny=8192, nz=1), lbm.LBM_ERR_INVALID_ARG),   # 27 nx ny >= 2^31
])
def test_create_rejects_bad_parameters(lib, kw, code):
    h = ctypes.c_void_p()
    assert lib.lbm3_create(ctypes.byref(_params(**kw)), None, ctypes.byref(h)) == code
    assert not h.value


def test_create_rejects_fast_uniform_velocity(lib):
    p = _params()
    p.u[1] = 0.5
    h = ctypes.c_void_p()
    assert lib.lbm3_create(ctypes.byref(p), None, ctypes.byref(h)) == lbm.LBM_ERR_INVALID_ARG


def test_null_arguments(lib):
    assert lib.lbm3_params_default(None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3_velocities(None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm3_get_step(None) == -1
    lib.lbm3_destroy(None)

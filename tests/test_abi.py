"""CPU checks of the C ABI: the library builds, loads and exports every symbol
include/lbm.h declares; struct layouts agree between C and the binding;
parameter validation answers before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2504_09024_gb300 import build as B
from paper_2504_09024_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:lbm|surr)_[a-z_]+)\s*\(", text)))


def test_header_functions_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", B.SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT ((?:lbm|surr)_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(lbm.SIGNATURES) == names


def test_struct_layout_matches_header(lib):
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(lbm_params), offsetof(lbm_params, u_wall),
         offsetof(lbm_params, fext_y), sizeof(lbm_diag), offsetof(lbm_diag, nonfinite),
         offsetof(lbm_diag, status));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    P, D = lbm.lbm_params, lbm.lbm_diag
    assert vals == [ctypes.sizeof(P), P.u_wall.offset, P.fext_y.offset, ctypes.sizeof(D),
                    D.nonfinite.offset, D.status.offset]


def test_defaults_and_strerror(lib):
    p = lbm.lbm_params_default()
    assert p.W == 4.0 and p.phi_a == 1.0 and abs(p.zeta - 1 / 6) < 1e-15 and p.dtype == lbm.LBM_F32
    for code in range(0, -10, -1):
        assert lbm.lbm_strerror(code) != "unknown error"


@pytest.mark.parametrize("field,value,code", [
    ("nx", 2, lbm.LBM_ERR_INVALID_ARG),
    ("walls_y", 3, lbm.LBM_ERR_INVALID_ARG),
    ("M_phi", 0.0, lbm.LBM_ERR_RATE),
    ("D_s", -1.0, lbm.LBM_ERR_RATE),
    ("nu_a", 0.0, lbm.LBM_ERR_RATE),
    ("W", 0.0, lbm.LBM_ERR_INVALID_ARG),
    ("reserved", 1, lbm.LBM_ERR_INVALID_ARG),
    ("dtype", 7, lbm.LBM_ERR_INVALID_ARG),
])
def test_validation_before_device_work(lib, field, value, code):
    p = lbm.lbm_params_default()
    p.nx, p.ny = 32, 16
    setattr(p, field, value)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == code
    assert not h.value


def test_null_context_calls(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_get_step(None) == -1
    assert lib.lbm_synchronize(None) == lbm.LBM_ERR_INVALID_ARG
    lib.lbm_destroy(None)

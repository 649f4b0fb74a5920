"""16-bit population storage (FP16 / BF16 deviations, FP32 collision) against
the FP64 oracle, through the C ABI.

Bounds (relative L2 of phi, Gamma and the velocity vector): 1e-3 with FP16
storage, 5e-3 with BF16 storage, the bounds the precision target states for
the 2048x1024 drop after 5000 steps, applied here to the smaller workloads
after 1000 steps (the full-size comparison is tests/test_zy_precision_full.py).
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2504_09024_gb300 import lbm, workloads as W
from parity import TOL, rel, vrel

pytestmark = pytest.mark.gpu

BOUND = {lbm.LBM_F16S: 1e-3, lbm.LBM_BF16S: 5e-3}
DTYPES = [lbm.LBM_F16S, lbm.LBM_BF16S]


def run(case, dtype, steps, kernel=lbm.LBM_KERNEL_AUTO):
    s = lbm.Sim(case.phys, dtype=dtype, kernel=kernel)
    s.init(case.phi, case.c, case.ux, case.uy, case.P)
    s.step(steps)
    return s


def errors(got, ref, with_u=True):
    e = {"phi": rel(got["phi"], ref["phi"]), "c": rel(got["c"], ref["c"])}
    if with_u:
        e["u"] = vrel(got, ref)  # the velocity vector, both components
    return e


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("which", ["lively", "512x256"])
def test_coupled_1000_steps(dtype, which):
    case = W.lively_shear_drop() if which == "lively" else W.shear_drop_512x256(steps=1000)
    ref = oracle.run_case(case, steps=1000).fields()
    e = errors(run(case, dtype, 1000).fields(), ref)
    assert max(e.values()) <= BOUND[dtype], e


@pytest.mark.parametrize("dtype", DTYPES)
def test_two_cells_per_thread(dtype):
    """16-bit storage with two cells per thread (packed FP32 arithmetic) on a
    ragged grid, against the oracle at the storage bound."""
    case = W.lively_shear_drop(nx=203, ny=61, R=14.0)
    ref = oracle.run_case(case, steps=600).fields()
    for shape in ((128, 32), (192, 24)):
        s = lbm.Sim(case.phys, dtype=dtype)
        s.set_launch_shape(*shape)
        s.set_cells_per_thread(2)
        s.init(case.phi, case.c, case.ux, case.uy)
        s.step(600)
        e = errors(s.fields(), ref)
        assert max(e.values()) <= BOUND[dtype], (shape, e)


@pytest.mark.parametrize("dtype", DTYPES)
def test_fixed_velocity_static_drop_1000_steps(dtype):
    case = W.static_drop_cos_mode()
    ref = oracle.run_case(case, steps=1000).fields()
    e = errors(run(case, dtype, 1000).fields(), ref, with_u=False)
    assert max(e.values()) <= BOUND[dtype], e


@pytest.mark.parametrize("dtype", DTYPES)
def test_conservation(dtype):
    """The zeroth moments stay in fixed point: sum phi and sum Gamma drift
    only by the rounding of the per-cell increments."""
    case = W.static_drop_cos_mode()
    s = lbm.Sim(case.phys, dtype=dtype)
    s.init(case.phi, case.c, case.ux, case.uy)
    d0 = s.diagnostics()
    s.step(2000)
    d1 = s.diagnostics()
    assert abs(d1["sum_phi"] - d0["sum_phi"]) < 1e-6 * d0["sum_phi"]
    assert abs(d1["sum_c"] - d0["sum_c"]) < 1e-5 * d0["sum_c"]


@pytest.mark.parametrize("dtype", DTYPES)
def test_initial_populations_rounded(dtype):
    """Packing rounds only the deviations: the populations after
    initialisation differ from the FP32 state by at most the 16-bit rounding
    of the shifted values (half a unit in the last place)."""
    case = W.lively_shear_drop()
    a = run(case, lbm.LBM_F32, 0).pops()
    b = run(case, dtype, 0).pops()
    ulp = 2.0 ** -11 if dtype == lbm.LBM_F16S else 2.0 ** -8
    for k in ("f", "h", "g"):
        shifted = np.abs(a[k]).max()
        assert np.abs(a[k] - b[k]).max() <= ulp * shifted, k


@pytest.mark.parametrize("dtype", DTYPES)
def test_graph_replay_equals_single_steps(dtype):
    """The stochastic rounding draws from (step, cell): a captured 32-step
    graph and single launches give the same bits."""
    case = W.lively_shear_drop()
    a = run(case, dtype, 40).pops()
    s = lbm.Sim(case.phys, dtype=dtype)
    s.init(case.phi, case.c, case.ux, case.uy)
    for _ in range(40):
        s.step(1)
    b = s.pops()
    for k in ("f", "h", "g"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("dtype", DTYPES)
def test_checkpoint_resume_bit_exact(dtype):
    case = W.lively_shear_drop()
    a = run(case, dtype, 200).pops()
    s = run(case, dtype, 100)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        s.save(path)
        s.close()
        t = lbm.Sim(case.phys, dtype=dtype)
        t.load(path)
        assert t.t == 100
        t.step(100)
        b = t.pops()
    for k in ("f", "h", "g"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("dtype", DTYPES)
def test_block_widths_agree_bitwise(dtype):
    """The per-cell arithmetic and the stochastic rounding's draws depend on
    (step, cell) only: 128- and 192-wide blocks give the same bits on a ragged
    grid."""
    case = W.lively_shear_drop(nx=203, ny=61, R=14.0)
    out = []
    for shape in ((128, 32), (192, 24)):
        s = lbm.Sim(case.phys, dtype=dtype)
        s.set_launch_shape(*shape)
        s.init(case.phi, case.c, case.ux, case.uy)
        s.step(150)
        out.append(s.pops())
    for k in ("f", "h", "g"):
        np.testing.assert_array_equal(out[0][k], out[1][k], err_msg=k)


def test_storage_options_rejected():
    case = W.lively_shear_drop()
    with pytest.raises(lbm.LBMError) as e:
        lbm.Sim(case.phys, dtype=lbm.LBM_F16S, kernel=lbm.LBM_KERNEL_FUSED)
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED
    s = lbm.Sim(case.phys, dtype=lbm.LBM_BF16S)
    with pytest.raises(lbm.LBMError) as e:
        s.set_launch_shape(64, 32)
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([case.phys], dtype=lbm.LBM_F16S)
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("dtype", DTYPES)
def test_autotune_restores_state(dtype):
    case = W.lively_shear_drop()
    s = run(case, dtype, 5)
    before = s.pops()
    tx, seg, ms = s.autotune(steps=4)
    assert tx in (128, 192) and seg >= 4 and ms > 0 and s.t == 5
    after = s.pops()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    ref = run(case, dtype, 45)
    s.step(40)
    np.testing.assert_array_equal(s.pops()["f"], ref.pops()["f"])


@pytest.mark.parametrize("dtype", [lbm.LBM_F16S, lbm.LBM_BF16S])
@pytest.mark.parametrize("shape,cpt", [((192, 32), 1), ((128, 24), 2), ((128, 5), 1)])
def test_16bit_store_modes_give_the_same_bits(dtype, shape, cpt):
    """16-bit storage written by direct stores or through the staging area
    and bulk-tensor stores: the same words land in the same places (a ragged
    grid with walls, so tail columns and ghost copies are exercised)."""
    case = W.lively_shear_drop(nx=131, ny=45, R=10.0)
    out = {}
    for mode in (lbm.LBM_STORE_DIRECT, lbm.LBM_STORE_STAGED):
        s = lbm.Sim(case.phys, dtype=dtype, kernel=lbm.LBM_KERNEL_TMA)
        s.set_launch_shape(*shape)
        s.set_cells_per_thread(cpt)
        s.set_store_mode(mode)
        s.init(case.phi, case.c, case.ux, case.uy)
        s.step(60)
        out[mode] = s.pops()
        s.close()
    for k in out[lbm.LBM_STORE_DIRECT]:
        np.testing.assert_array_equal(out[lbm.LBM_STORE_DIRECT][k], out[lbm.LBM_STORE_STAGED][k],
                                      err_msg=k)

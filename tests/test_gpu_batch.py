"""Batched runs and the launch-shape autotuner, through the C ABI.

A batched step runs the same per-cell arithmetic as a single run's TMA sweep,
so with equal launch shapes every run of a batch must match, bit for bit, the
same run stepped on its own; one batch is also held to the FP64 oracle at the
single-run bounds of the lively drop.  The autotuner must leave the state, the step count and
the buffer parity as it found them.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2504_09024_gb300 import lbm, workloads as W
from parity import check_lively

pytestmark = pytest.mark.gpu



def mixed_cases():
    """Uneven grids and parameters: the ragged lively drop, a shrunken
    ensemble draw of each grid class, and a periodic-y variant."""
    draws = W.ensemble_draws(nruns=6, seed=77)
    cases = [W.lively_shear_drop()]
    cases += [W.ensemble_case(d, shrink=4) for d in draws[:3]]
    small = W.lively_shear_drop(nx=72, ny=44, R=10.0)
    periodic = dataclasses.replace(small.phys, walls_y=0, u_wall=0.0)
    cases.append(dataclasses.replace(small, name="periodic_drop", phys=periodic,
                                     ux=np.zeros_like(small.ux), uy=np.zeros_like(small.uy)))
    return cases


def init_all(sims, cases):
    for s, c in zip(sims, cases):
        s.init(c.phi, c.c, c.ux, c.uy, c.P)


P_, C_ = lbm.LBM_BATCH_PERSISTENT, lbm.LBM_BATCH_CHAINS
D_, S_ = lbm.LBM_STORE_DIRECT, lbm.LBM_STORE_STAGED


@pytest.mark.parametrize("shape,cpt,out,form", [
    ((128, 32), 1, D_, P_), ((64, 16), 1, S_, P_), ((192, 24), 2, D_, P_), ((192, 24), 2, S_, P_),
    ((128, 32), 2, S_, C_), ((192, 24), 1, D_, C_)])
def test_batch_bitwise_equals_single_runs(shape, cpt, out, form):
    cases = mixed_cases()
    b = lbm.Batch([c.phys for c in cases])
    b.set_form(form)
    b.set_launch_shape(*shape)
    b.set_cells_per_thread(cpt)
    b.set_store_mode(out)
    init_all(b.runs, cases)
    singles = [lbm.Sim(c.phys, kernel=lbm.LBM_KERNEL_TMA) for c in cases]
    for s in singles:
        s.set_launch_shape(*shape)
        s.set_cells_per_thread(cpt)
        s.set_store_mode(out)
    init_all(singles, cases)
    b.step(70)  # graphs of 32, 32, 4 and 2 steps
    b.sync()
    for s in singles:
        s.step(70)
    for k, (r, s) in enumerate(zip(b.runs, singles)):
        assert r.t == s.t == 70
        fr, fs = r.fields(), s.fields()
        for key in ("phi", "c", "ux", "uy", "P"):
            np.testing.assert_array_equal(fr[key], fs[key], err_msg=f"run {k} {key}")
    b.close()


def test_batch_matches_oracle_1000_steps():
    cases = [W.lively_shear_drop(), W.lively_shear_drop(nx=130, ny=60)]
    b = lbm.Batch([c.phys for c in cases])
    init_all(b.runs, cases)
    b.step(1000)
    b.sync()
    for r, c in zip(b.runs, cases):
        check_lively(r.fields(), oracle.run_case(c, steps=1000).fields(), oracle, c, 1000)
    b.close()


def test_run_stepped_alone_rejoins_batch():
    """A run stepped on its own (odd count: its buffer parity flips) is picked
    up by the next batched step."""
    cases = mixed_cases()[:3]
    b = lbm.Batch([c.phys for c in cases])
    init_all(b.runs, cases)
    singles = [lbm.Sim(c.phys, kernel=lbm.LBM_KERNEL_TMA) for c in cases]
    init_all(singles, cases)
    b.runs[1].step(3)
    singles[1].step(3)
    b.step(5)
    b.sync()
    for s in singles:
        s.step(5)
    assert [r.t for r in b.runs] == [5, 8, 5]
    for r, s in zip(b.runs, singles):
        np.testing.assert_array_equal(r.fields()["phi"], s.fields()["phi"])
        np.testing.assert_array_equal(r.fields()["ux"], s.fields()["ux"])
    b.close()


def test_batch_launch_shape_and_tiles():
    cases = mixed_cases()
    b = lbm.Batch([c.phys for c in cases])
    for tx, seg in ((128, 32), (64, 48), (128, 4), (192, 16)):
        b.set_launch_shape(tx, seg)
        bx, sy, blocks, tiles = b.launch_shape()
        expect = sum(-(-c.phys.nx // (tx - 4)) * -(-c.phys.ny // seg) for c in cases)
        assert (bx, sy, tiles) == (tx, seg, expect)
        assert 1 <= blocks <= tiles
    with pytest.raises(lbm.LBMError):
        b.set_launch_shape(96, 32)
    with pytest.raises(lbm.LBMError):
        b.set_launch_shape(128, 2)
    b.close()


def test_batch_rejects_mixed_modes():
    a = W.lively_shear_drop().phys
    fixed = W.static_drop_cos_mode().phys
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, fixed])


def test_batch_stall_hook_reports_timeout():
    cases = mixed_cases()[:2]
    b = lbm.Batch([c.phys for c in cases])
    init_all(b.runs, cases)
    lbm.lbm_debug_stall_next_step(b.runs[1].ctx)
    b.step(1)
    with pytest.raises(lbm.LBMError) as ei:
        b.sync()
    assert ei.value.code == lbm.LBM_ERR_TIMEOUT
    # usable again after re-initialisation
    init_all(b.runs, cases)
    b.step(40)
    b.sync()
    for r in b.runs:
        assert np.isfinite(r.fields()["phi"]).all()
    b.close()


def test_autotune_single_restores_state():
    case = W.lively_shear_drop()
    s = lbm.Sim(case.phys, kernel=lbm.LBM_KERNEL_TMA)
    s.init(case.phi, case.c, case.ux, case.uy, case.P)
    s.step(7)
    before = s.fields()
    tx, seg, ms = s.autotune(steps=8)
    assert tx in (64, 128, 192) and seg >= 4 and ms > 0
    assert lbm.lbm_get_launch_shape(s.ctx) == (tx, seg)
    assert s.cells_per_thread in (1, 2)
    assert s.t == 7
    after = s.fields()
    for k in before:
        np.testing.assert_array_equal(before[k], after[k])
    # stepping on continues exactly as an untuned run with the chosen shape
    ref = lbm.Sim(case.phys, kernel=lbm.LBM_KERNEL_TMA)
    ref.set_launch_shape(tx, seg)
    ref.set_cells_per_thread(s.cells_per_thread)
    ref.set_store_mode(s.store_mode)
    ref.init(case.phi, case.c, case.ux, case.uy, case.P)
    ref.step(7 + 40)
    s.step(40)
    np.testing.assert_array_equal(s.fields()["phi"], ref.fields()["phi"])


def test_batch_autotune_restores_state():
    cases = mixed_cases()
    b = lbm.Batch([c.phys for c in cases])
    init_all(b.runs, cases)
    b.step(5)
    b.sync()
    before = [r.fields() for r in b.runs]
    tx, seg, ms = b.autotune(steps=4)
    assert tx in (64, 128, 192) and seg >= 4 and ms > 0
    assert b.launch_shape()[:2] == (tx, seg)
    assert b.form in (lbm.LBM_BATCH_CHAINS, lbm.LBM_BATCH_PERSISTENT)
    assert [r.t for r in b.runs] == [5] * len(cases)
    for r, f0 in zip(b.runs, before):
        f1 = r.fields()
        for k in f0:
            np.testing.assert_array_equal(f0[k], f1[k])
    b.close()


@pytest.mark.parametrize("form", [P_, C_])
@pytest.mark.parametrize("shape,cpt,out", [((192, 32), 1, D_), ((128, 24), 1, S_),
                                           ((128, 24), 2, D_)])
def test_nonfinite_run_leaves_other_runs_unchanged(form, shape, cpt, out):
    """A run whose state turns non-finite (here a NaN in its initial phi)
    changes no bit of the other runs of its batch: runs of one batch share
    blocks, shared memory and parameter slots, never data."""
    good = W.lively_shear_drop(nx=131, ny=45, R=10.0)
    other = W.ensemble_case(W.ensemble_draws(nruns=2, seed=5)[0], shrink=4)
    bad_phi = good.phi.copy()
    bad_phi[20:24, 60:70] = np.nan
    cases = [good, dataclasses.replace(good, name="bad", phi=bad_phi), other, good]
    b = lbm.Batch([c.phys for c in cases])
    b.set_form(form)
    b.set_launch_shape(*shape)
    b.set_cells_per_thread(cpt)
    b.set_store_mode(out)
    init_all(b.runs, cases)
    b.step(40)
    b.sync()
    assert b.runs[1].diagnostics()["nonfinite"] > 0
    for k in (0, 2, 3):
        s = lbm.Sim(cases[k].phys, kernel=lbm.LBM_KERNEL_TMA)
        s.set_launch_shape(*shape)
        s.set_cells_per_thread(cpt)
        s.set_store_mode(out)
        s.init(cases[k].phi, cases[k].c, cases[k].ux, cases[k].uy, cases[k].P)
        s.step(40)
        fr, fs = b.runs[k].fields(), s.fields()
        for key in ("phi", "c", "ux", "uy", "P"):
            np.testing.assert_array_equal(fr[key], fs[key], err_msg=f"run {k} {key}")
        s.close()
    b.close()

"""The allocation-free statistics entry point against lbm_diagnostics.

lbm_field_stats_noalloc serves callers that cannot allocate device memory
where they need the statistics; its scratch is a static device array shared
by every call.  Two calls in a row, on two different states, must each give
the same numbers as the allocating entry point.  This file is collected last
so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

from paper_2504_09024_gb300 import lbm, workloads as W

pytestmark = pytest.mark.gpu

KEYS = [(0, "sum_phi"), (1, "sum_c"), (2, "xc"), (3, "yc"), (4, "nonfinite"),
        (5, "sigma_neg"), (6, "umax"), (10, "L"), (11, "B"), (12, "D")]


def test_field_stats_noalloc_matches_diagnostics():
    import torch
    case = W.lively_shear_drop()
    p = case.phys
    sim = lbm.Sim(p)
    sim.init(case.phi, case.c, case.ux, case.uy)
    fields = [torch.empty((p.ny, p.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
    result = torch.full((lbm.LBM_FIELD_STATS_LEN,), float("nan"), dtype=torch.float64,
                        device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for steps in (150, 250):  # two calls in a row, on two different states
        sim.step(steps)
        ref = sim.diagnostics()
        lbm.lbm_get_fields_device(sim.ctx, *fields)
        sim.sync()
        lbm.lbm_field_stats_noalloc(*fields, p.nx, p.ny, p.walls_y, p.beta, p.c_max, result,
                                    stream, phi_a=p.phi_a, phi_b=p.phi_b)
        torch.cuda.synchronize()
        got = result.cpu().numpy()
        for k, name in KEYS:
            assert abs(got[k] - ref[name]) <= 1e-12 * max(1.0, abs(ref[name])), (steps, name)
        # other bulk phases: phi mapped affinely onto (phi_b, phi_a) = (-1, 2)
        # has the same drop indicator, so the same centroid and shape
        mapped = [fields[0] * 3.0 - 1.0] + fields[1:]
        lbm.lbm_field_stats_noalloc(*mapped, p.nx, p.ny, p.walls_y, p.beta, p.c_max, result,
                                    stream, phi_a=2.0, phi_b=-1.0)
        torch.cuda.synchronize()
        got = result.cpu().numpy()
        for k, name in KEYS:
            if name in ("xc", "yc", "L", "B", "D"):
                assert abs(got[k] - ref[name]) <= 1e-9 * max(1.0, abs(ref[name])), (steps, name)
    sim.close()


def test_field_stats_noalloc_rejects_bad_sizes():
    import torch
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    r = torch.zeros(lbm.LBM_FIELD_STATS_LEN, dtype=torch.float64, device="cuda")
    for nx, ny in ((0, 4), (4, 0), (1 << 16, 1 << 15)):
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_field_stats_noalloc(x, x, x, x, nx, ny, 0, 0.0, 1.0, r)
        assert e.value.code == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LBMError) as e:  # equal bulk phases
        lbm.lbm_field_stats_noalloc(x, x, x, x, 2, 2, 0, 0.0, 1.0, r, phi_a=0.5, phi_b=0.5)
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG

"""Host-side pieces of the Table 1 driver (Sec. 4.3): the Stone-Leal
small-deformation formula at its closed-form limits, and the run set-up."""
import math

import pytest

from paper_2504_09024_gb300 import table1 as T


@pytest.mark.parametrize("Ca", [0.01, 0.03, 0.05])
def test_stone_leal_clean_is_taylor_limit(Ca):
    # beta = 0, lambda = 1: b_r = (5/4)(35/20) = 35/16, independent of Pe
    b = 35.0 / 16.0
    for Pe in (0.1, 10.0, 1e6):
        assert math.isclose(T.stone_leal(Ca, 0.0, Pe), 3 * Ca * b / (4 + Ca * b), rel_tol=1e-14)
    # small Ca: D -> (3/4) b_r Ca
    assert math.isclose(T.stone_leal(1e-9, 0.0, 1.0) / 1e-9, 0.75 * b, rel_tol=1e-6)


def test_stone_leal_surfactant_limits():
    # Pe/Ca -> infinity: b_r -> (5/4)(4/2) = 5/2 for any beta > 0
    assert math.isclose(T.stone_leal(0.02, 0.25, 1e12), 3 * 0.02 * 2.5 / (4 + 0.02 * 2.5), rel_tol=1e-9)
    # surfactant raises D at every Ca (the trend Sec. 4.3 reports)
    for Ca in T.TABLE1:
        assert T.stone_leal(Ca, 0.25, 10.0) > T.stone_leal(Ca, 0.0, 10.0)


def test_table1_cases_follow_the_setup():
    cases = T.make_cases()
    assert len(cases) == 2 * len(T.TABLE1)
    for c in cases:
        H = c.phys.ny
        assert (c.phys.nx, H) == (768, 256) and c.meta["R"] == H / 8
        gd = c.meta["gamma_dot"]
        assert math.isclose(gd * c.meta["R"] ** 2 / T.NU, 0.1, rel_tol=1e-12)        # Re
        assert math.isclose(T.NU * gd * c.meta["R"] / c.phys.sigma_o, c.meta["Ca"], rel_tol=1e-12)
        assert math.isclose(c.phys.u_wall * c.phys.W / c.phys.M_phi, 0.5, rel_tol=1e-12)  # Pe*
        assert math.isclose(2 * c.phys.u_wall / H, gd, rel_tol=1e-12)

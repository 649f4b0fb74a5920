"""Control logic of the surrogate-guided Ca_crit search on the host: the
LBM labelling is replaced by a known breakup boundary (breakup iff
Ca > 0.15 + 0.4 beta), so every decision of verify / fallback / bisection
can be checked without a GPU."""
import numpy as np
import pytest

from paper_2504_09024_gb300 import sweep


def truth(pts):
    return 0.15 + 0.4 * np.asarray(pts["beta"])


@pytest.fixture
def fake_lbm(monkeypatch):
    calls = []

    def labels(pts, grid, t_star=sweep.T_STAR, batch=512, samples=5):
        ca = np.asarray(pts["Ca"], dtype=float)
        calls.append(len(ca))
        brk = ca > truth(pts)
        D = 0.5 * ca
        return D, brk, np.ones(len(ca), dtype=bool), len(ca) * 100

    monkeypatch.setattr(sweep, "lbm_labels", labels)
    return calls


def test_bad_predictions_end_with_lbm_ca_crit(fake_lbm):
    pts = sweep.draw_points(6, seed=3)
    pts["beta"] = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.25])
    t = truth(pts)
    pred = t.copy()
    pred[1] = np.nan           # the network gave no Ca
    pred[2] = t[2] + 0.2       # far too high: the lower check run breaks up
    pred[3] = t[3] - 0.15      # far too low: the upper check run stays whole
    pred[4] = t[4] + 0.07      # off by more than the bracket
    ca, source, counts = sweep.resolve(pts, pred, (32, 16))
    assert np.all(np.isfinite(ca))
    # confirmed predictions are kept as they are
    assert source.tolist() == [1, 0, 0, 0, 0, 1]
    assert ca[0] == pred[0] and ca[5] == pred[5]
    # every LBM result lies within half the final bracket width of the boundary
    assert np.all(np.abs(ca - t) <= sweep.BRACKET + 1e-12), np.abs(ca - t)
    assert counts["confirmed"] == 2
    assert counts["verify_runs"] == 2 * 5          # two runs per finite prediction
    assert counts["fallback_points"] == 4
    assert counts["fallback_runs"] > 0


def test_fallback_brackets_follow_the_check_runs():
    pred = np.array([0.3, 0.3, 0.3, np.nan, 0.3])
    confirmed = np.array([True, False, False, False, False])
    brk_lo = np.array([False, True, False, False, True])
    brk_hi = np.array([True, True, False, False, False])
    idx, lo, hi = sweep.fallback_brackets(pred, confirmed, brk_lo, brk_hi)
    assert idx.tolist() == [1, 2, 3, 4]
    # 1: the run at 0.25 broke up -> below it
    assert (lo[0], hi[0]) == (sweep.CA_RANGE[0], pytest.approx(0.25))
    # 2: the run at 0.35 stayed whole -> above it
    assert (lo[1], hi[1]) == (pytest.approx(0.35), sweep.CA_RANGE[1])
    # 3: no prediction, 4: both outcomes contradict the prediction -> anywhere
    assert (lo[2], hi[2]) == sweep.CA_RANGE and (lo[3], hi[3]) == sweep.CA_RANGE


def test_bisection_from_brackets_runs_only_open_points(fake_lbm):
    pts = sweep.draw_points(3, seed=4)
    pts["beta"] = np.array([0.1, 0.2, 0.3])
    lo = np.array([0.05, 0.2, 0.2])
    hi = np.array([0.5, 0.3, 0.5])     # the second bracket is already closed
    ca, runs, _ = sweep.lbm_bisection(pts, (32, 16), lo=lo, hi=hi)
    assert abs(ca[1] - 0.25) < 1e-12
    assert np.all(np.abs(ca - truth(pts)) <= sweep.BRACKET + 1e-12)
    assert runs == sum(fake_lbm)
    assert all(n <= 2 for n in fake_lbm)   # the closed bracket is never run


def test_aspect_is_a_live_input():
    pts = sweep.draw_points(256, seed=1)
    a = pts["aspect"]
    assert a.min() >= sweep.ASPECT_RANGE[0] and a.max() <= sweep.ASPECT_RANGE[1]
    assert a.std() > 0.02
    X = sweep.features(pts)
    assert np.all(np.abs(X[:, 4]) <= 1.0 + 1e-6) and X[:, 4].std() > 0.3
    # every run of a grid has the same shear rate, so the same steps reach t*
    g = (384, 128)
    rates = []
    for asp in (0.2, 0.25, 0.3):
        R = sweep.radius(asp, g)
        case = sweep.make_case(0.2, 0.1, 10.0, 0.3, asp, g)
        rates.append(case.meta["gamma_dot"])
        assert abs(case.meta["R"] - R) < 1e-12
    assert max(rates) - min(rates) < 1e-12 * max(rates)

"""The surrogate-guided critical-Ca search, end to end on toy-sized runs,
and the Ca_crit bisection on a network trained to a known boundary."""
import numpy as np
import pytest

from paper_2504_09024_gb300 import lbm, sweep

pytestmark = pytest.mark.gpu


def test_bisection_finds_a_known_boundary():
    """Train the network (GPU kernels) on labels with breakup iff
    Ca > 0.15 + 0.4 beta, then recover the boundary by bisection."""
    pts = sweep.draw_points(4096, seed=5)
    yB = (pts["Ca"] > 0.15 + 0.4 * pts["beta"]).astype(np.float32)
    yD = (0.5 * pts["Ca"]).astype(np.float32)
    net, loss = sweep.train_surrogate(sweep.features(pts), yD, yB, epochs=1500, lr=3e-3)
    q = sweep.draw_points(64, seed=6)
    ca = sweep.predict_ca_crit(net, q)
    truth = 0.15 + 0.4 * q["beta"]
    inside = truth < sweep.CA_RANGE[1] - 0.02
    assert np.all(np.isfinite(ca[inside]))
    assert np.max(np.abs(ca[inside] - truth[inside])) < 0.03, np.abs(ca - truth)
    net.close()


def test_sweep_pipeline_small():
    rep = sweep.main(["--grid", "96x32", "--train", "48", "--heldout", "8", "--points", "8",
                      "--baseline-points", "4", "--t-star", "0.3", "--epochs", "300"])
    assert rep["train_runs"] == 48 and rep["sweep_points"] == 8
    assert rep["heldout_points"] == 8 and 0.0 <= rep["heldout_breakup_accuracy"] <= 1.0
    assert rep["verify_runs"] == 2 * rep["predicted"]
    # every point ends with a Ca_crit: confirmed, or found by the LBM fallback
    assert rep["resolved"] == rep["sweep_points"]
    assert rep["fallback_points"] == rep["sweep_points"] - rep["confirmed"]
    assert rep["runs_per_point_with_surrogate"] == pytest.approx(
        (rep["verify_runs"] + rep["fallback_runs"]) / rep["sweep_points"])
    # from [0.05, 0.5] to a bracket 0.1 wide: three LBM runs per point
    assert rep["baseline_runs"] == 3 * 4
    assert rep["runs_per_hour"] > 0
    assert rep["gpu_hours_surrogate_with_training"] >= rep["gpu_hours_surrogate_search"] > 0

"""The JSONL metrics log on the host, with a stand-in run (no GPU)."""
import json

from paper_2504_09024_gb300 import lbm, metrics


class FakeSim:
    nx, ny = 64, 32
    mode = lbm.LBM_COUPLED
    cells_per_thread = 1
    store_mode = 0

    def __init__(self):
        self.params = lbm.lbm_params()
        self.params.nx, self.params.ny, self.params.dtype = 64, 32, lbm.LBM_F32
        self.t = 0
        self.ctx = None

    def sync(self):
        pass

    def diagnostics(self):
        return {"sum_phi": 100.0 + self.t, "sum_c": 5.0, "D": 0.1, "L": 12.0, "B": 9.0,
                "nonfinite": 0}


def test_metrics_log_lines(tmp_path, monkeypatch):
    monkeypatch.setattr(lbm, "lbm_get_launch_shape", lambda ctx: (192, 38))
    sim = FakeSim()
    path = tmp_path / "run.jsonl"
    log = metrics.MetricsLog(str(path), sim, run="r0", extra={"Ca": 0.2})
    log.record()
    sim.t = 1000
    log.record(note="second")
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) == 2
    a, b = lines
    assert a["run"] == "r0" and a["step"] == 0 and a["params"]["nx"] == 64 and a["Ca"] == 0.2
    assert "MLUPS" not in a and "params" not in b
    assert b["step"] == 1000 and b["sum_phi"] == 1100.0 and b["note"] == "second"
    assert b["MLUPS"] > 0 and abs(b["GBps"] - b["MLUPS"] * 216 / 1000) <= 1e-9 * b["GBps"]
    assert b["dtype"] == "f32" and b["launch_shape"] == [192, 38]


def test_bytes_per_cell():
    assert metrics.bytes_per_cell(lbm.LBM_F32, True) == 216
    assert metrics.bytes_per_cell(lbm.LBM_F16S, True) == 108
    assert metrics.bytes_per_cell(lbm.LBM_F32, False) == 144

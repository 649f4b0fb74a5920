"""Multi-rank aggregation of bench.py (replicas: every rank times its own
grid; the job value is all ranks' cell updates over the slowest rank's time),
run as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench = load_bench()
    local_ms = [120.0, 150.0][rank]
    ms_max = bench.max_over_ranks(local_ms, dist, device="cpu")
    value = bench.whole_job_mlups(world, 2_097_152, 1000, ms_max * 1e-3)
    out.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    expect = 2 * 2_097_152 * 1000 / 0.150 / 1e6
    assert all(abs(r[2] - expect) < 1e-6 * expect for r in res)


def test_single_rank_is_identity():
    bench = load_bench()
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_mlups(1, 100, 10, 0.5) == 100 * 10 / 0.5 / 1e6

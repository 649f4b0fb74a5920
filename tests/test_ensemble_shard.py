"""One ensemble sharded over ranks (every run stepped by exactly one rank,
per-run diagnostics gathered to rank 0), with two gloo ranks on the CPU.
The runs are stepped by the FP64 oracle here (the GPU path steps each rank's
runs as one lbm.Batch); the sharding and gathering are the same code."""
import os
import socket

import numpy as np
import pytest

from paper_2504_09024_gb300 import ensemble, workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("sum_phi", "sum_c", "D", "L", "B")
STEPS = 20


def tiny_cases(n=5):
    draws = W.ensemble_draws(nruns=n, seed=W.CASE_SEED)
    return [W.ensemble_case(d, shrink=16, steps=STEPS) for d in draws]


def step_runs(orc, cases, runs):
    rows = {}
    for r in runs:
        c = cases[r]
        s = orc.Sim(c.phys)
        s.init(c.phi, c.c, c.ux, c.uy, None)
        s.step(STEPS)
        d = s.diagnostics()
        rows[r] = [float(d[k]) for k in KEYS]
        s.close()
    return rows


def test_shard_deals_every_run_once():
    rng = np.random.default_rng(3)
    for n, world in ((1, 1), (5, 2), (64, 4), (7, 8)):
        cells = rng.integers(1, 10_000, n)
        owned = ensemble.shard(cells, world)
        assert len(owned) == world
        flat = sorted(r for o in owned for r in o)
        assert flat == list(range(n))
        loads = [int(sum(cells[r] for r in o)) for o in owned]
        assert max(loads) - min(loads) <= int(cells.max())


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cases = tiny_cases()
    owned = ensemble.shard([c.phys.nx * c.phys.ny for c in cases], world)[rank]
    rows = step_runs(oracle, cases, owned)
    merged = ensemble.gather_rows(rows, dist)
    out.put((rank, owned, merged))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cases = tiny_cases()
    (_, own0, merged), (_, own1, none) = res
    assert none is None
    assert sorted(own0 + own1) == list(range(len(cases))) and not set(own0) & set(own1)
    single = step_runs(oracle_mod, cases, range(len(cases)))
    assert sorted(merged) == sorted(single)
    for r in single:
        assert merged[r] == single[r], r

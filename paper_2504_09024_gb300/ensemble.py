"""Sharding one ensemble of independent runs over the ranks of a job.

The runs of an ensemble share nothing, so a job of N ranks (one GPU each)
steps disjoint subsets of them and needs no collective in the data path:
the runs are dealt out by cell count (largest first, each to the rank with
the fewest cells so far), every rank steps its own runs as one batch, and
the per-run diagnostics are gathered to rank 0 at the end.  This module holds
only that host logic; the stepping is the caller's (lbm.Batch on a GPU).
"""
from __future__ import annotations


def shard(cells, world: int):
    """Run indices per rank: runs in decreasing cell count, each to the rank
    with the fewest cells so far (ties to the lower rank), so every run is
    owned by exactly one rank and the loads differ by at most one run."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda r: (-int(cells[r]), r))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda q: (load[q], q))
        owned[k].append(r)
        load[k] += int(cells[r])
    return [sorted(o) for o in owned]


def gather_rows(rows, dist=None):
    """Per-run rows of every rank, gathered to rank 0: `rows` maps a run index
    to a list of numbers.  Returns the merged dict on rank 0 (and on every
    rank of a single-process job), None elsewhere.  A run reported by two
    ranks is an error."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return dict(rows)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(rows))
    if dist.get_rank() != 0:
        return None
    merged = {}
    for part in parts:
        for run, row in part.items():
            if run in merged:
                raise RuntimeError(f"run {run} reported by two ranks")
            merged[run] = row
    return merged

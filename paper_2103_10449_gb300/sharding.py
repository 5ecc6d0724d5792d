"""Replica sharding across ranks (host logic, no device work).

Switching realisations and dCCI pairs are independent units; the two phases of a pair stay
together because they exchange (U, V) every step.  One process per GPU takes a contiguous
range of units balanced by atom count; the only collectives are after the run: the maximum
of the timed intervals and a gather of per-unit results.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard_units(atoms_per_unit: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Contiguous [start, end) unit ranges, one per rank, balancing the atom count: rank r
    takes the units whose cumulative atom count (at their midpoint) falls in the r-th
    1/world of the total.  Every unit is assigned exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = len(atoms_per_unit)
    total = float(sum(atoms_per_unit))
    bounds = [0] * (world + 1)
    bounds[world] = n
    if total <= 0 or n == 0:
        for r in range(world + 1):
            bounds[r] = min(n, (n * r) // world)
        return [(bounds[r], bounds[r + 1]) for r in range(world)]
    acc = 0.0
    r = 1
    for u, a in enumerate(atoms_per_unit):
        mid = acc + 0.5 * a
        while r < world and mid >= total * r / world:
            bounds[r] = u
            r += 1
        acc += a
    while r < world:
        bounds[r] = n
        r += 1
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def rank_seed(base: int, rank: int) -> int:
    """Distinct, reproducible noise seeds per rank (rank 0 keeps the base seed)."""
    return base + 7919 * rank


def aggregate_throughput(units_done_per_rank: Sequence[float], wall_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return float(sum(units_done_per_rank)) / wall_max


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over the process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(rows: list, dist=None) -> list:
    """All ranks' per-unit result rows (rank order) on every rank."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return list(rows)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, list(rows))
    merged = []
    for part in out:
        merged.extend(part)
    return merged


def run_sharded(atoms_per_unit: Sequence[int], rank: int, world: int, build, warmup: int, steps: int,
                md_steps_per_step: int, dist=None, device=None, barrier=None, before_timed=None,
                after_timed=None) -> dict:
    """One rank's part of a replica job, the orchestration the benchmark runs on every rank.

    The units (independent replicas or dCCI pairs, ``atoms_per_unit`` atoms each) are split by
    ``shard_units``; ``build(lo, hi)`` returns this rank's engine for units [lo, hi), an object
    with ``warmup(k)``, ``timed(k)`` (seconds of k timed steps, measured on the device) and
    ``rows()`` (one result row per unit).  The timed region is bracketed by ``barrier`` (and
    ``before_timed`` / ``after_timed``, e.g. a clock sampler); afterwards the slowest rank's time,
    the whole-job throughput (atom-steps of all ranks over that time) and every unit's result
    row (all-gathered, in unit order) are returned.  No collective runs inside the timed region."""
    lo, hi = shard_units(atoms_per_unit, world)[rank]
    eng = build(lo, hi)
    eng.warmup(warmup)
    if barrier is not None:
        barrier()
    if before_timed is not None:
        before_timed()
    wall = eng.timed(steps)
    if barrier is not None:
        barrier()
    if after_timed is not None:
        after_timed()
    wall_max = max_over_ranks(wall, dist, device)
    mine = float(sum(atoms_per_unit[lo:hi])) * md_steps_per_step * steps
    done = gather_results([mine], dist)
    return {"value": aggregate_throughput(done, wall_max), "wall": wall, "wall_max": wall_max,
            "range": (lo, hi), "atom_steps_per_rank": done, "rows": gather_results(eng.rows(), dist),
            "engine": eng}

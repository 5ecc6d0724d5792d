"""Multi-rank host logic on CPU (gloo, world size 2): replica sharding, max-over-ranks timing,
whole-job throughput and the final gather of results."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2103_10449_gb300 import inputs as I
from paper_2103_10449_gb300 import sharding as S


def test_shard_units_covers_each_unit_once_and_balances_atoms():
    sizes = [int(s) for s in I.log_uniform_sizes(64, 512, 32768, seed=3)]
    for world in (1, 2, 3, 4, 8):
        parts = S.shard_units(sizes, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(sizes)
        assert all(a <= b for a, b in parts) and all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        loads = [sum(sizes[a:b]) for a, b in parts]
        assert sum(loads) == sum(sizes)
        assert max(loads) - min(loads) <= max(sizes) * 1.01 + 1
    assert S.shard_units([], 3) == [(0, 0), (0, 0), (0, 0)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [8000] * 10 + [512, 32768]
    lo, hi = S.shard_units(sizes, world)[rank]
    atoms = sum(sizes[lo:hi])
    wall = 1.0 + rank                        # rank 1 is the slow one
    wmax = S.max_over_ranks(wall, dist)
    done = [float(atoms * 32 * 10)]
    every = [None] * world
    dist.all_gather_object(every, done[0])
    value = S.aggregate_throughput(every, wmax)
    rows = S.gather_results([(u, sizes[u]) for u in range(lo, hi)], dist)
    if rank == 0:
        out.put((wmax, value, rows, S.rank_seed(1000, 1)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_timing_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    wmax, value, rows, seed1 = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sizes = [8000] * 10 + [512, 32768]
    assert wmax == 2.0
    assert value == pytest.approx(sum(sizes) * 32 * 10 / 2.0)
    assert [u for u, _ in rows] == list(range(len(sizes)))
    assert seed1 == 1000 + 7919


class _StubEngine:
    """Host stand-in for a rank's engine (no device): 'timed' reports a fixed duration that
    differs by rank, 'rows' one result per unit."""

    def __init__(self, lo, hi, rank):
        self.lo, self.hi, self.rank = lo, hi, rank
        self.warm = 0

    def warmup(self, k):
        self.warm = k

    def timed(self, k):
        return 0.5 * k * (1 + self.rank)

    def rows(self):
        return [(u, 2.0 * u, self.rank) for u in range(self.lo, self.hi)]


def _orchestration_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [int(s) for s in I.log_uniform_sizes(64, 512, 32768, seed=2021)]
    calls = []
    res = S.run_sharded(sizes, rank, world, lambda lo, hi: _StubEngine(lo, hi, rank), 3, 4, 32, dist=dist,
                        barrier=dist.barrier, before_timed=lambda: calls.append("before"),
                        after_timed=lambda: calls.append("after"))
    if rank == 0:
        out.put((res["value"], res["wall_max"], res["rows"], res["range"], res["atom_steps_per_rank"], calls,
                 res["engine"].warm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_runs_the_benchmark_orchestration():
    """sharding.run_sharded, the function bench.py runs on every rank (for the replica benchmark
    and the batched dCCI pairs), with a host stub engine: the units are split by atom count, the
    slowest rank's time is the job's time, the throughput counts every rank's atom-steps, and every
    unit's result row comes back in unit order."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_orchestration_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    value, wall_max, rows, rng, per_rank, calls, warm = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sizes = [int(s) for s in I.log_uniform_sizes(64, 512, 32768, seed=2021)]
    parts = S.shard_units(sizes, 2)
    assert rng == parts[0] and warm == 3 and calls == ["before", "after"]
    assert wall_max == 0.5 * 4 * 2                       # rank 1 is the slower one
    assert per_rank == [float(sum(sizes[a:b])) * 32 * 4 for a, b in parts]
    assert value == pytest.approx(sum(sizes) * 32 * 4 / wall_max)
    assert [r[0] for r in rows] == list(range(len(sizes)))
    assert [r[2] for r in rows] == [0] * (parts[0][1] - parts[0][0]) + [1] * (parts[1][1] - parts[1][0])

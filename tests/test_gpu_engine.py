"""Engine runs on the GPU: long-run stability of batched replicas and conservation checks.

The per-system error word must stay clear (no NaN, no list or cell inconsistency), the
thermostat must hold the temperature, and the list must keep every in-cutoff pair.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KB = 8.617333262e-5
MVV2E = 1.66053906660e-23 / 1.602176634e-19


def _ctx(N, nrep, T=1000.0, precision=0, nsched=20000):
    x, box = I.diamond(10, 10, 10)
    sv = math.sqrt(KB * T / (28.0855 * MVV2E))
    ctx = N.Context(precision=precision, skin=0.5, nbr_cap=48)
    for r in range(nrep):
        s = ctx.add_system(x, box, v=I.gaussian_velocities(len(x), sv, 50 + r), r0=x)
        ctx.set_thermostat(s, T, 0.1, 50 + r)
        ctx.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if r % 2 == 0 else -1, nsteps=nsched, k_E=5.0)
    return ctx, len(x)


def test_batched_frenkel_ladd_long_run_stays_physical():
    from paper_2103_10449_gb300 import nefe as N
    ctx, n = _ctx(N, 6)
    ctx.run(4000)
    res = ctx.results_all()
    for r in res:
        assert r["error"] == 0, r
        assert 800.0 < r["T"] < 1200.0, r["T"]
        assert math.isfinite(r["W"]) and math.isfinite(r["U"])
    # forward replicas are SW diamond: cohesive energy near -4.34 + 3/2 kT at 1000 K
    u = [r["U"] / n for i, r in enumerate(res) if i % 2 == 0]
    assert all(-4.30 < e < -4.10 for e in u), u
    mean_row, max_row, builds = ctx.list_stats(-1)
    assert 15.0 < mean_row < 20.0 and max_row <= 48
    ctx.close()


def test_rebuild_all_policy_rebuilds_together_and_keeps_forces_exact():
    """Policy rebuild_all: on a step where one system's list is stale every system rebuilds.
    The systems then count the same builds, more than under the per-system policy, and the
    engine's SW energy of each final state equals the oracle's brute-force energy of it."""
    from oracle import oracle as O
    from paper_2103_10449_gb300 import nefe as N
    builds = {}
    for pol in (0, 1):
        ctx, n = _ctx(N, 3, precision=0)
        ctx.set_tuning(0)
        ctx.set_rebuild_policy(pol)
        ctx.run(400)
        builds[pol] = [ctx.list_stats(s)[2] for s in range(3)]
        if pol == 1:
            for s in range(3):
                x, _, box = ctx.get_state(s)
                r = ctx.results(s)
                assert r["error"] == 0
                assert r["U"] == pytest.approx(O.sw_energy(x, box)[0], rel=1e-5)
        ctx.close()
    assert len(set(builds[1])) == 1 and builds[1][0] > 5
    assert builds[1][0] >= max(builds[0])


def test_list_holds_every_pair_inside_the_cutoff_after_a_long_run():
    """Verlet guarantee: each pair closer than a*sigma at the current positions is in the
    engine's list.  The engine's SW energy of the state it reports after 2000 steps must equal
    the FP64 oracle's brute-force energy of that same state (O(N^2), no list at all): a pair
    missing from a row would drop its terms from the engine's U."""
    from oracle import oracle as O
    from paper_2103_10449_gb300 import nefe as N
    ctx, n = _ctx(N, 1, precision=1)
    ctx.run(2000)
    x, v, box = ctx.get_state(0)
    r = ctx.results(0)
    ctx.close()
    e_o = O.sw_energy(x, box)[0]
    assert r["U"] == pytest.approx(e_o, rel=1e-10)


_DEBUG_RUN = r"""
import sys, math
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2103_10449_gb300 import inputs as I, nefe as N
x, box = I.diamond(3, 3, 3)
sv = math.sqrt(8.617333262e-5 * 1000.0 / (28.0855 * 1.66053906660e-23 / 1.602176634e-19))
ctx = N.Context(precision=N.NEFE_FP32, skin=0.5, nbr_cap=48)
s = ctx.add_system(x, box, v=I.gaussian_velocities(len(x), sv, 71), r0=x)
ctx.set_thermostat(s, 1000.0, 0.1, 72)
ctx.set_schedule(s, N.NEFE_SCHED_FL, nsteps=400, k_E=5.0)
ctx.set_tuning(0)
ctx.run(101)
r = ctx.results(s)
xs, _, _ = ctx.get_state(s)
print(N._build.LIB_DEBUG if N.load()._name.endswith("libnefe_debug.so") else N._build.LIB)
print(repr(r["W"]), r["error"], repr(float(np.abs(xs).sum())))
"""


def test_debug_bounds_build_runs_the_same_trajectory():
    """libnefe_debug.so (index checks on every atom index read from device data) runs a scatter-
    form switching run bit for bit like the normal library and raises no error bit."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for flag in ("0", "1"):
        env = dict(os.environ, NEFE_DEBUG_BOUNDS=flag)
        p = subprocess.run([sys.executable, "-c", _DEBUG_RUN, root], env=env, capture_output=True, text=True,
                           timeout=900)
        assert p.returncode == 0, p.stderr[-2000:]
        lib, vals = p.stdout.strip().splitlines()[-2:]
        assert lib.endswith("libnefe_debug.so" if flag == "1" else "libnefe.so")
        out[flag] = vals.split()
    assert out["0"] == out["1"]
    assert out["1"][1] == "0"


def test_cooperative_rebuild_builds_the_same_lists():
    """The list rebuild as one cooperative launch (worklist, cells and lists between grid
    barriers) and as the kernel sequence build the same lists, so the runs are bit for bit equal
    -- under both rebuild policies, with rebuilds along the way."""
    from paper_2103_10449_gb300 import nefe as N
    for pol in (0, 1):
        out = []
        for coop in (0, 1):
            ctx, n = _ctx(N, 3, precision=0)
            ctx.set_tuning(0, None, 0)
            ctx.set_rebuild_policy(pol)
            ctx.set_cooperative_rebuild(coop)
            ctx.run(200)
            ctx.sync()
            out.append(([ctx.results(s)["W"] for s in range(3)], [ctx.get_state(s)[0] for s in range(3)],
                        ctx.list_stats(-1)[2]))
            assert all(r["error"] == 0 for r in ctx.results_all())
            ctx.close()
        (wa, xa, ba), (wb, xb, bb) = out
        assert ba == bb and ba > 5
        assert wa == wb and all(np.array_equal(p, q) for p, q in zip(xa, xb))


def test_grid_barrier_gives_up_by_its_time_limit():
    """Failure detection of the one device-side wait (the grid barriers of the single-launch list
    rebuild): a barrier that can never complete must end every waiting block by its limit and
    report NEFE_ETIMEOUT; the device stays usable (an engine run afterwards is error free)."""
    import time
    from paper_2103_10449_gb300 import nefe as N
    t0 = time.perf_counter()
    rc = N.nefe_check_barrier_timeout(0, 50.0)
    assert rc == N.NEFE_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    ctx, n = _ctx(N, 2, precision=0)
    ctx.run(64)
    ctx.sync()
    assert all(r["error"] == 0 for r in ctx.results_all())
    ctx.close()

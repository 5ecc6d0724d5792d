"""Batching of uneven systems in one context (FP64 kernels) against the oracle, system by system.

One context holds two dCCI pairs of different sizes (temperature and pressure control), a backward
Frenkel-Ladd replica and a reversible-scaling NPT replica — 6 systems of 64 to 216 atoms, so tiles of
several systems share launches and the per-system sums, schedules and pair updates must stay apart.
Each system (or pair) is compared with its own oracle run: positions within 1e-8 A, work and the
coexistence estimates within 1e-8 relative after 80 steps (the FP64 trajectory parity of the single-system
tests).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GPA = O.EV_A3_TO_GPA
NST = 80


def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


@pytest.mark.parametrize("rebuild_all", [0, 1])
def test_uneven_batch_matches_oracle_per_system(N, rebuild_all):
    """With rebuild_all every system rebuilds its list on a step where any system needs one: the
    lists are then rebuilt earlier than needed, which must leave every trajectory on the oracle's
    (which has no list at all), and every system counts the same builds."""
    T = 400.0
    p0 = 10.0
    xa1, ba1 = I.diamond(2, 2, 2)
    xb1, bb1 = I.beta_tin(2, 2, 4)
    xa2, ba2 = I.diamond(3, 3, 3)
    xb2, bb2 = I.beta_tin(3, 3, 6)
    xf, bf = I.diamond(3, 3, 3)
    xr, br = I.diamond(2, 2, 2)
    pos = [xa1, xb1, xa2, xb2, xf, xr]
    boxes = [ba1, bb1, ba2, bb2, bf, br]
    vel = [I.gaussian_velocities(len(x), _sv(T), 100 + k) for k, x in enumerate(pos)]
    seeds = [200 + k for k in range(len(pos))]

    ctx = N.Context(precision=N.NEFE_FP64)
    ids = [ctx.add_system(pos[k], boxes[k], v=vel[k], r0=pos[k] if k == 4 else None) for k in range(len(pos))]
    assert ids == list(range(len(pos)))
    for k in range(len(pos)):
        ctx.set_thermostat(k, T, 0.1, seeds[k])
    for a, b in ((0, 1), (2, 3)):
        ctx.set_barostat(a, N.NEFE_BARO_ISO, p0, 0.5)
        ctx.set_barostat(b, N.NEFE_BARO_ANISO, p0, 0.5)
    pid_t = ctx.pair_dcci(0, 1, T, p0, N.NEFE_DCCI_TEMP, T, 500.0, 200)
    pid_p = ctx.pair_dcci(2, 3, T, p0, N.NEFE_DCCI_PRESS, p0, 12.0, 150)
    ctx.set_schedule(4, N.NEFE_SCHED_FL, direction=-1, nsteps=300, k_E=5.0)
    ctx.set_barostat(5, N.NEFE_BARO_ISO, 1.0, 0.5)
    ctx.set_schedule(5, N.NEFE_SCHED_RS, nsteps=200, lambda_f=0.5, P_GPa=1.0)
    ctx.set_rebuild_policy(rebuild_all)
    ctx.run(NST)
    res = ctx.results_all()
    states = [ctx.get_state(k) for k in range(len(pos))]
    pairs = [ctx.pair(pid_t), ctx.pair(pid_p)]
    builds = [ctx.list_stats(k)[2] for k in range(len(pos))]
    assert ctx.rebuild_policy() == rebuild_all
    ctx.close()
    assert all(r["error"] == 0 for r in res)
    if rebuild_all:
        assert len(set(builds)) == 1 and builds[0] >= 1, builds

    def sysk(k, **kw):
        return O.System(x=pos[k].copy(), v=vel[k].copy(), box=boxes[k].copy(), T=T, tdamp=0.1, seed=seeds[k],
                        sys_id=k, **kw)

    # dCCI pairs
    for (a, b, mode, frm, to, nsched), got in zip(((0, 1, O.DCCI_TEMP, T, 500.0, 200),
                                                   (2, 3, O.DCCI_PRESS, p0 / GPA, 12.0 / GPA, 150)), pairs):
        sa = sysk(a, baro=O.BARO_ISO, pdamp=0.5)
        sb = sysk(b, baro=O.BARO_ANISO, pdamp=0.5)
        pr = O.DcciPair(sa, sb, T, p0 / GPA, mode, frm, to, nsched)
        pr.run(NST)
        T_c, P_c, lam, err = got
        To, Po = pr.coexistence()
        assert err == 0 and pr.error == 0
        assert lam == pytest.approx(pr.lam, rel=1e-8)
        assert T_c == pytest.approx(To, rel=1e-8)
        assert P_c == pytest.approx(Po * GPA, rel=1e-7, abs=1e-9)
        assert np.abs(states[a][0] - sa.x).max() < 1e-8
        assert np.abs(states[b][0] - sb.x).max() < 1e-8
    # backward Frenkel-Ladd replica
    of = sysk(4, r0=pos[4].copy(), k_E=5.0, sched=O.SCHED_FL, direction=-1, nsched=300).run(NST)
    assert res[4]["W"] == pytest.approx(of.W, rel=1e-8, abs=1e-9)
    assert np.abs(states[4][0] - of.x).max() < 1e-8
    # reversible scaling, NPT
    orr = sysk(5, baro=O.BARO_ISO, p_ext=1.0 / GPA, pdamp=0.5, sched=O.SCHED_RS, nsched=200, lam_f=0.5).run(NST)
    assert res[5]["W"] == pytest.approx(orr.W, rel=1e-8)
    assert np.abs(states[5][0] - orr.x).max() < 1e-8
    assert np.allclose(states[5][2], orr.box, rtol=1e-11, atol=0)

"""Switching protocols on the GPU against the FP64 oracle, through the C ABI.

Reversible scaling with the lambda-scaled barostat (Sec. 2.2), adiabatic switching in
pressure (Sec. 2.3), the coupled dCCI pair in temperature and pressure control (Sec. 3), and
the harmonic-crystal switching whose free energy is known in closed form (Sec. 2.1).
The FP64 kernels must follow the oracle's trajectory step for step (tolerances of a few
1e-9 relative: the summation order differs, and chaos amplifies it over ~100 steps).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GPA = O.EV_A3_TO_GPA


def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


def test_reversible_scaling_npt_matches_oracle(N):
    x0, box = I.diamond(2, 2, 2)
    v0 = I.gaussian_velocities(len(x0), _sv(400.0), 3)
    nst, nsched, P = 120, 200, 1.0
    orc = O.System(x=x0.copy(), v=v0.copy(), box=box.copy(), T=400.0, tdamp=0.1, seed=4, sys_id=0,
                   baro=O.BARO_ISO, p_ext=P / GPA, pdamp=0.5, sched=O.SCHED_RS, nsched=nsched, lam_f=0.5)
    orc.run(nst)
    ctx = N.Context(precision=N.NEFE_FP64)
    s = ctx.add_system(x0, box, v=v0)
    ctx.set_thermostat(s, 400.0, 0.1, 4)
    ctx.set_barostat(s, N.NEFE_BARO_ISO, P, 0.5)
    ctx.set_schedule(s, N.NEFE_SCHED_RS, nsteps=nsched, lambda_f=0.5, P_GPa=P)
    ctx.run(nst)
    r = ctx.results(s)
    x, v, b = ctx.get_state(s)
    ctx.close()
    ro = orc.results()
    assert r["lambda"] == pytest.approx(ro["lam"], rel=1e-14)
    assert np.allclose(b, ro["box"], rtol=1e-11, atol=0)
    assert r["V"] == pytest.approx(ro["V"], rel=1e-11)
    assert np.abs(x - orc.x).max() < 1e-8
    assert r["W"] == pytest.approx(ro["W"], rel=1e-8)
    assert r["U"] == pytest.approx(ro["U"], rel=1e-9)
    assert np.allclose(r["P"], ro["P"], rtol=1e-6, atol=1e-6)
    assert r["P_target"] == pytest.approx(ro["lam"] * P, rel=1e-12)


def test_pressure_switching_matches_oracle(N):
    x0, box = I.beta_tin(2, 2, 4)
    v0 = I.gaussian_velocities(len(x0), _sv(400.0), 5)
    nst = 100
    orc = O.System(x=x0.copy(), v=v0.copy(), box=box.copy(), T=400.0, tdamp=0.1, seed=6, sys_id=0,
                   baro=O.BARO_ANISO, pdamp=0.5, sched=O.SCHED_AS, nsched=150, p0=10.0 / GPA,
                   p1=12.0 / GPA)
    orc.run(nst)
    ctx = N.Context(precision=N.NEFE_FP64)
    s = ctx.add_system(x0, box, v=v0)
    ctx.set_thermostat(s, 400.0, 0.1, 6)
    ctx.set_barostat(s, N.NEFE_BARO_ANISO, 10.0, 0.5)
    ctx.set_schedule(s, N.NEFE_SCHED_AS, nsteps=150, P0_GPa=10.0, P1_GPa=12.0)
    ctx.run(nst)
    r = ctx.results(s)
    x, v, b = ctx.get_state(s)
    ctx.close()
    ro = orc.results()
    assert r["lambda"] == pytest.approx(ro["lam"] * GPA, rel=1e-12)
    assert np.allclose(b, ro["box"], rtol=1e-11, atol=0)
    assert np.abs(x - orc.x).max() < 1e-8
    assert r["W"] == pytest.approx(ro["W"], rel=1e-8)


@pytest.mark.parametrize("mode", ["temp", "press"])
def test_dcci_pair_matches_oracle(N, mode):
    xa, ba = I.diamond(2, 2, 2)
    xb, bb = I.beta_tin(2, 2, 4)
    va = I.gaussian_velocities(len(xa), _sv(400.0), 7)
    vb = I.gaussian_velocities(len(xb), _sv(400.0), 8)
    p0 = 10.0
    if mode == "temp":
        omode, nmode, frm, to = O.DCCI_TEMP, N.NEFE_DCCI_TEMP, 400.0, 500.0
        ofrm, oto = frm, to
    else:
        omode, nmode, frm, to = O.DCCI_PRESS, N.NEFE_DCCI_PRESS, p0, 12.0
        ofrm, oto = frm / GPA, to / GPA
    nst, nsched = 80, 200
    a = O.System(x=xa.copy(), v=va.copy(), box=ba.copy(), tdamp=0.1, seed=9, sys_id=0,
                 baro=O.BARO_ISO, pdamp=0.5)
    b = O.System(x=xb.copy(), v=vb.copy(), box=bb.copy(), tdamp=0.1, seed=9, sys_id=1,
                 baro=O.BARO_ANISO, pdamp=0.5)
    pair = O.DcciPair(a, b, 400.0, p0 / GPA, omode, ofrm, oto, nsched)
    pair.run(nst)
    ctx = N.Context(precision=N.NEFE_FP64)
    sa = ctx.add_system(xa, ba, v=va)
    sb = ctx.add_system(xb, bb, v=vb)
    for s in (sa, sb):
        ctx.set_thermostat(s, 400.0, 0.1, 9)
    ctx.set_barostat(sa, N.NEFE_BARO_ISO, p0, 0.5)
    ctx.set_barostat(sb, N.NEFE_BARO_ANISO, p0, 0.5)
    pid = ctx.pair_dcci(sa, sb, 400.0, p0, nmode, frm, to, nsched)
    ctx.run(nst)
    T_c, P_c, lam, err = ctx.pair(pid)
    xg, _, _ = ctx.get_state(sa)
    ctx.close()
    To, Po = pair.coexistence()
    assert err == 0 and pair.error == 0
    assert lam == pytest.approx(pair.lam, rel=1e-9)
    assert T_c == pytest.approx(To, rel=1e-9)
    assert P_c == pytest.approx(Po * GPA, rel=1e-7, abs=1e-9)
    assert np.abs(xg - a.x).max() < 1e-8


def _equilibrated(N, pot_k, T, seed, nrep, steps=800):
    """nrep 64-atom Einstein crystals (spring pot_k about the lattice) equilibrated at T."""
    x0, box = I.diamond(2, 2, 2)
    ctx = N.Context(precision=N.NEFE_FP32)
    for r in range(nrep):
        s = ctx.add_system(x0, box, v=I.gaussian_velocities(len(x0), _sv(T), seed + r), r0=x0,
                           pot=N.NEFE_POT_EINSTEIN, k_int=pot_k)
        ctx.set_thermostat(s, T, 0.1, seed + r)
    ctx.run(steps)
    states = [ctx.get_state(r)[:2] for r in range(nrep)]
    ctx.close()
    return x0, box, states


def test_harmonic_switching_on_gpu_reproduces_closed_form(N):
    """Einstein k=5 <-> k=10 at 400 K: 1/2 (W_f - W_b)/N = 3/2 kB T ln 2 within 1 meV/atom
    (the closed form of the classical harmonic crystal; the FP32 kernels)."""
    T, nrep, nsw = 400.0, 16, 2000
    x0, box, fwd = _equilibrated(N, 5.0, T, 100, nrep)
    _, _, bwd = _equilibrated(N, 10.0, T, 300, nrep)
    ctx = N.Context(precision=N.NEFE_FP32)
    ids = []
    for r in range(nrep):
        for direction, st in ((1, fwd[r]), (-1, bwd[r])):
            s = ctx.add_system(st[0], box, v=st[1], r0=x0, pot=N.NEFE_POT_EINSTEIN, k_int=5.0)
            ctx.set_thermostat(s, T, 0.1, 1000 + 2 * r + (direction < 0))
            ctx.set_schedule(s, N.NEFE_SCHED_FL, direction=direction, nsteps=nsw, k_E=10.0)
            ids.append((s, direction))
    ctx.run(nsw)
    res = ctx.results_all()
    ctx.close()
    wf = [res[s]["W"] for s, d in ids if d > 0]
    wb = [res[s]["W"] for s, d in ids if d < 0]
    assert all(r["error"] == 0 for r in res)
    dF = 0.5 * (np.mean(wf) - np.mean(wb)) / len(x0)
    assert abs(dF - 1.5 * O.KB * T * math.log(2.0)) < 1e-3


def test_checkpoint_resume_is_bitwise(N, tmp_path):
    x0, box = I.diamond(3, 3, 3)
    v0 = I.gaussian_velocities(len(x0), _sv(600.0), 11)

    def make():
        ctx = N.Context(precision=N.NEFE_FP32)
        s = ctx.add_system(x0, box, v=v0, r0=x0)
        ctx.set_thermostat(s, 600.0, 0.1, 12)
        ctx.set_schedule(s, N.NEFE_SCHED_FL, nsteps=500, k_E=5.0)
        return ctx
    ref = make()
    ref.run(300)
    r_ref = ref.results(0)
    x_ref, v_ref, _ = ref.get_state(0)
    ref.close()
    a = make()
    a.run(120)
    a.save(tmp_path / "ck.bin")
    a.close()
    b = make()
    b.setup()
    b.load(tmp_path / "ck.bin")
    b.run(180)
    r = b.results(0)
    x, v, _ = b.get_state(0)
    b.close()
    assert r["W"] == r_ref["W"] and r["step"] == 300
    assert np.array_equal(x, x_ref) and np.array_equal(v, v_ref)

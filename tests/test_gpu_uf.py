"""The Uhlenbeck-Ford fluid reference on the GPU (through the C ABI) against the FP64 oracle.

The liquid's free energy in the paper (Sec. 2.1, Sec. 4) comes from Hamiltonian interpolation
between liquid SW silicon and the UF fluid (p = 25, sigma = 2.0 A at 2200 K); the UF fluid's own
free energy is computed here by switching from the ideal gas.  Tolerances as for the SW kernels:
energies, per-atom energies and forces (normwise) within 1e-10 (FP64 kernel) or 1e-5 (FP32
kernel) of the oracle; trajectories of the FP64 path within 1e-8 A and 1e-8 of W.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UF = (25.0, 2.0, 2200.0, 8.0)      # p, sigma (A), T_uf (K), rc (A)
SKIN = 0.5
RCS = O.SW_SI[6] * O.SW_SI[1] + SKIN


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


def soa(x):
    return torch.tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=torch.float64, device="cuda")


def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


def configs():
    out = {}
    x, b = I.liquid(1500, 0.05, seed=31, rmin=1.6)
    out["fluid1500"] = (x + np.array([-50.0, 7.0, 130.0]), b)        # unwrapped, 11 tiles + 92
    n = 700
    L = (n / 0.05) ** (1.0 / 3.0)
    out["ideal700"] = (np.random.default_rng(32).uniform(0.0, L, (n, 3)), np.array([L, L, L]))   # close pairs
    return out


CONFIGS = configs()


def _uf_forces(N, x, box, precision):
    n = len(x)
    f = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    ea = torch.zeros(n, dtype=torch.float64, device="cuda")
    ev = torch.zeros(7, dtype=torch.float64, device="cuda")
    N.nefe_uf_forces(soa(x), n, box, RCS, SKIN, N.uf_params(*UF), precision, f, ea, ev)
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(3, n).T, ea.cpu().numpy(), ev.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("name", list(CONFIGS))
def test_uf_energy_forces_virial(N, name, precision, tol):
    x, box = CONFIGS[name]
    e_o, f_o, vir_o, ea_o = O.uf_energy(x, box, UF)
    f, ea, ev = _uf_forces(N, x, box, precision)
    assert np.abs(f - f_o).max() <= tol * np.abs(f_o).max()
    assert abs(ev[0] - e_o) <= tol * abs(e_o)
    assert np.abs(ea - ea_o).max() <= tol * np.abs(ea_o).max()
    assert np.abs(ev[1:] - vir_o).max() <= tol * np.abs(vir_o).max() * 10


def test_uf_forces_bitwise_reproducible_and_checked(N):
    x, box = CONFIGS["fluid1500"]
    a = _uf_forces(N, x, box, 0)
    b = _uf_forces(N, x, box, 0)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    n = len(x)
    f = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    with pytest.raises(N.NefeError):                           # fewer than 5 cells per axis
        N.nefe_uf_forces(soa(x), n, np.array([20.0, 40.0, 40.0]), RCS, SKIN, N.uf_params(*UF), 0, f)
    with pytest.raises(N.NefeError):                           # rc + skin above 2 rcs
        N.nefe_uf_forces(soa(x), n, box, RCS, SKIN, N.uf_params(rc=9.0), 0, f)


def _fluid(n, rho, seed, rmin=1.9):
    x, b = I.liquid(n, rho, seed=seed, rmin=rmin)
    return x, b


def _pair_run(N, precision, kind, nsteps, nsched=400):
    """One engine system and the oracle, same start and noise: 'ideal' switches the ideal gas
    to the UF fluid (FL interpolation with the UF reference), 'liquid' switches SW atoms to the
    UF fluid, 'uf' runs the UF fluid at fixed lambda (NVT)."""
    T = UF[2]
    x0, box = _fluid(600, 0.05, seed=41)
    v0 = I.gaussian_velocities(len(x0), _sv(T), 42)
    kw = dict(x=x0.copy(), v=v0.copy(), box=box.copy(), r0=x0.copy(), uf=UF, T=T, tdamp=0.1, seed=43, sys_id=0)
    if kind == "ideal":
        orc = O.System(pot=O.POT_EINSTEIN, k_int=0.0, ref=O.REF_UF, sched=O.SCHED_FL, nsched=nsched, **kw)
    elif kind == "liquid":
        orc = O.System(pot=O.POT_SW, ref=O.REF_UF, sched=O.SCHED_FL, nsched=nsched, **kw)
    else:
        orc = O.System(pot=O.POT_UF, **kw)
    orc.run(nsteps)
    ctx = N.Context(precision=precision, skin=SKIN, nbr_cap=48)
    if kind == "ideal":
        s = ctx.add_system(x0, box, v=v0, r0=x0, pot=N.NEFE_POT_EINSTEIN, k_int=0.0)
    elif kind == "liquid":
        s = ctx.add_system(x0, box, v=v0, r0=x0)
    else:
        s = ctx.add_system(x0, box, v=v0, r0=x0, pot=N.NEFE_POT_UF)
    ctx.set_uf_params(s, N.uf_params(*UF))
    ctx.set_thermostat(s, T, 0.1, 43)
    if kind != "uf":
        ctx.set_schedule(s, N.NEFE_SCHED_FL, direction=1, nsteps=nsched, ref=N.NEFE_REF_UF)
    ctx.run(nsteps)
    res = ctx.results(s)
    x, v, _ = ctx.get_state(s)
    ctx.close()
    return orc, res, x, v


@pytest.mark.parametrize("kind", ["ideal", "liquid", "uf"])
def test_uf_trajectory_fp64_matches_oracle(N, kind):
    orc, res, x, v = _pair_run(N, 1, kind, 120)
    ro = orc.results()
    assert res["error"] == 0
    assert np.abs(x - orc.x).max() < 1e-8
    assert res["U"] == pytest.approx(ro["U"], rel=1e-9, abs=1e-9)
    assert res["U_E"] == pytest.approx(ro["U_E"], rel=1e-9, abs=1e-9)
    assert res["W"] == pytest.approx(ro["W"], rel=1e-8, abs=1e-9)
    assert res["T"] == pytest.approx(ro["T"], rel=1e-7)


@pytest.mark.parametrize("kind", ["ideal", "liquid"])
def test_uf_trajectory_fp32_close_to_oracle(N, kind):
    orc, res, x, v = _pair_run(N, 0, kind, 60)
    ro = orc.results()
    assert res["error"] == 0
    assert np.abs(x - orc.x).max() < 1e-4
    assert res["W"] == pytest.approx(ro["W"], rel=1e-4, abs=1e-4)


def test_uf_switching_run_is_bitwise_deterministic(N):
    a = _pair_run(N, 0, "liquid", 100)
    b = _pair_run(N, 0, "liquid", 100)
    assert a[1]["W"] == b[1]["W"] and np.array_equal(a[2], b[2])


def test_ideal_gas_to_uf_free_energy_follows_the_virial_series_on_gpu(N):
    """The same physics pin as the oracle's, at a size the oracle cannot run: 10 + 10 switches
    of 8000 atoms at rho B2 = 0.2, 20000 steps each, FP32 kernels; F_ex / (N kT) against
    (N-1)/N rho B2 + rho^2 B3 / 2 (the B4 term is about 0.4 % of the total at this density)."""
    n, target, reps, nsw = 8000, 0.2, 10, 20000
    p, sig, T = int(UF[0]), UF[1], UF[2]
    b2, b3 = O.uf_b2(p, sig), O.uf_b3(p, sig)
    rho = target / b2
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    # backward switches start from the UF fluid equilibrated at lambda = 1 (2 ps at 2200 K)
    eq = N.Context(precision=N.NEFE_FP32, skin=SKIN, nbr_cap=48)
    for r in range(reps):
        x = np.random.default_rng(800 + r).uniform(0.0, L, (n, 3))
        s = eq.add_system(x, box, v=I.gaussian_velocities(n, _sv(T), 900 + r), pot=N.NEFE_POT_UF)
        eq.set_uf_params(s, N.uf_params(*UF))
        eq.set_thermostat(s, T, 0.1, 950 + r)
    eq.run(2000)
    uf_states = [eq.get_state(s)[:2] for s in range(reps)]
    eq.close()
    ctx = N.Context(precision=N.NEFE_FP32, skin=SKIN, nbr_cap=48)
    fw, bw = [], []
    for r in range(2 * reps):
        if r < reps:       # the ideal gas: uniform positions are its equilibrium
            x = np.random.default_rng(500 + r).uniform(0.0, L, (n, 3))
            v = I.gaussian_velocities(n, _sv(T), 600 + r)
        else:
            x, v = uf_states[r - reps]
        s = ctx.add_system(x, box, v=v, r0=x, pot=N.NEFE_POT_EINSTEIN, k_int=0.0)
        ctx.set_uf_params(s, N.uf_params(*UF))
        ctx.set_thermostat(s, T, 0.1, 700 + r)
        fwd = r < reps
        ctx.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if fwd else -1, nsteps=nsw, ref=N.NEFE_REF_UF)
        (fw if fwd else bw).append(s)
    ctx.run(nsw)
    res = ctx.results_all()
    ctx.close()
    assert all(r["error"] == 0 for r in res)
    wf = np.array([res[s]["W"] for s in fw])
    wb = np.array([res[s]["W"] for s in bw])
    kT = O.KB * T
    fex = O.free_energy_difference(wf, wb) / (n * kT)
    sem = 0.5 * math.sqrt(wf.var(ddof=1) / reps + wb.var(ddof=1) / reps) / (n * kT)
    pred = (n - 1) / n * rho * b2 + rho ** 2 * b3 / 2.0
    assert sem < 2e-3
    assert abs(fex - pred) < 4.0 * sem + 0.003

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: neighbour lists and cells bit-exact; SW energy,
forces and virial within 1e-10 (FP64 kernel) or 1e-5 (FP32 kernel) relative, forces measured
normwise as max|dF| / max|F|; thermostat noise from the same Philox stream within 1e-14
(FP64 transform) / 2e-4 (FP32 transform on 24-bit uniforms, whose rounding the Box-Muller
radius sqrt(-2 ln u) amplifies in the tails).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = O.SW_SI[6] * O.SW_SI[1]
SKIN = 0.5
RCS = RC + SKIN
CAP = 48


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


def soa(x):
    return torch.tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=torch.float64, device="cuda")


def configs():
    out = {}
    x, b = I.diamond(2, 2, 2)
    out["diamond64"] = (I.rattle(x, 0.1, 1), b)                 # 2 cells per axis
    x, b = I.diamond(5, 5, 5)
    out["diamond1000"] = (I.rattle(x, 0.15, 2), b)              # 7 tiles + ragged 104
    x, b = I.beta_tin(6, 6, 12)
    out["betatin1728"] = (I.rattle(x, 0.1, 3), b)
    x, b = I.liquid(1500, 0.05425, seed=4)
    out["liquid1500"] = (x + np.array([60.0, -30.0, 0.5]), b)   # unwrapped coordinates
    return out


CONFIGS = configs()


def gpu_list(N, x, box, cap=CAP):
    n = len(x)
    xd = soa(x)
    nbr = torch.zeros(n * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    N.nefe_neighbor_build(xd, n, box, RCS, cap, nbr, cnt)
    torch.cuda.synchronize()
    return xd, nbr, cnt


@pytest.mark.parametrize("name", list(CONFIGS))
def test_cell_bin_bit_exact(N, name):
    x, box = CONFIGS[name]
    n = len(x)
    nc_o, cell_o, start_o, perm_o = O.cell_bin(x, box, RCS)
    xd = soa(x)
    cap = int(np.prod(nc_o))
    cell = torch.zeros(n, dtype=torch.int32, device="cuda")
    start = torch.zeros(cap + 1, dtype=torch.int32, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    nc = N.nefe_cell_bin(xd, n, box, RCS, cell, start, perm, cap)
    torch.cuda.synchronize()
    assert tuple(nc) == tuple(nc_o)
    assert np.array_equal(cell.cpu().numpy(), cell_o)
    assert np.array_equal(start.cpu().numpy(), start_o)
    assert np.array_equal(perm.cpu().numpy(), perm_o)


@pytest.mark.parametrize("name", list(CONFIGS))
def test_neighbor_list_bit_exact(N, name):
    x, box = CONFIGS[name]
    n = len(x)
    nbr_o, cnt_o, img_o = O.neighbor_list(x, box, RCS, cap=CAP)
    _, nbr, cnt = gpu_list(N, x, box)
    nbr = nbr.cpu().numpy().reshape(n, CAP)
    cnt = cnt.cpu().numpy()
    assert np.array_equal(cnt, cnt_o)
    for i in range(n):
        j = nbr[i, :cnt[i]] & N.INDEX_MASK
        assert np.array_equal(j, nbr_o[i, :cnt[i]])
    # the stored cell offsets reproduce the minimum-image displacement
    code = (nbr >> N.CODE_SHIFT) & 31
    o = np.stack([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1], axis=-1)
    nc = np.array([int(np.floor(box[k] / RCS)) for k in range(3)])
    for k in range(3):
        while box[k] / nc[k] < RCS * (1 + 1e-9):
            nc[k] -= 1
    h = box / nc
    s = x / box
    fl = np.floor(s)
    c = np.minimum(((s - fl) * nc).astype(int), nc - 1)
    q = fl.astype(int) * nc + c
    xs = x - q * h
    for i in range(0, n, max(1, n // 50)):
        jj = nbr[i, :cnt[i]] & N.INDEX_MASK
        d = xs[jj] - xs[i] + o[i, :cnt[i]] * h
        d_o = x[nbr_o[i, :cnt[i]]] - x[i] - img_o[i, :cnt[i]] * box
        assert np.abs(d - d_o).max() < 1e-9


def _forces(N, x, box, precision):
    n = len(x)
    xd, nbr, cnt = gpu_list(N, x, box)
    f = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    ea = torch.zeros(n, dtype=torch.float64, device="cuda")
    ev = torch.zeros(7, dtype=torch.float64, device="cuda")
    prm = N.params_from(O.SW_SI)
    N.nefe_sw_forces(xd, n, box, RCS, nbr, cnt, CAP, prm, precision, f, ea, ev)
    torch.cuda.synchronize()
    return f.cpu().numpy().reshape(3, n).T, ea.cpu().numpy(), ev.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-5)])
@pytest.mark.parametrize("name", list(CONFIGS))
def test_sw_energy_forces_virial(N, name, precision, tol):
    x, box = CONFIGS[name]
    e_o, f_o, vir_o, ea_o = O.sw_energy(x, box)
    f, ea, ev = _forces(N, x, box, precision)
    fscale = np.abs(f_o).max()
    assert np.abs(f - f_o).max() <= tol * fscale
    assert abs(ev[0] - e_o) <= tol * abs(e_o)
    assert np.abs(ea - ea_o).max() <= tol * np.abs(ea_o).max()
    vscale = np.abs(vir_o).max()
    assert np.abs(ev[1:] - vir_o).max() <= tol * vscale * 10


def test_sw_forces_deterministic(N):
    x, box = CONFIGS["liquid1500"]
    a = _forces(N, x, box, 0)
    b = _forces(N, x, box, 0)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("precision,tol", [(1, 1e-14), (0, 2e-4)])
def test_langevin_noise(N, precision, tol):
    n = 5000
    xi = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    N.nefe_langevin_noise(17, 3, 12345, n, precision, xi)
    torch.cuda.synchronize()
    got = xi.cpu().numpy().reshape(n, 3)
    ref = O.langevin_xi(17, 3, 12345, n)
    assert np.abs(got - ref).max() <= tol * max(1.0, np.abs(ref).max())


def test_neighbor_overflow_and_bad_box_are_errors(N):
    x, box = CONFIGS["liquid1500"]
    n = len(x)
    xd = soa(x)
    nbr = torch.zeros(n * 8, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    ovf = N.nefe_neighbor_build(xd, n, box, RCS, 8, nbr, cnt, check=False)
    assert ovf == 1
    with pytest.raises(N.NefeError):
        N.nefe_neighbor_build(xd, n, np.array([8.0, 8.0, 8.0]), RCS, CAP, nbr, cnt)
    # empty input is a no-op
    N.nefe_neighbor_build(xd, 0, box, RCS, CAP, nbr, cnt)


# ------------------------------------------------------------------ trajectories
def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


def _fl_pair(precision, nsteps=300, T=400.0, lanes=None, gather_lanes=None, list_lanes=None):
    x0, box = I.diamond(2, 2, 2)
    v0 = I.gaussian_velocities(len(x0), _sv(T), 1)
    orc = O.System(x=x0.copy(), v=v0.copy(), box=box.copy(), r0=x0.copy(), k_E=5.0, T=T, tdamp=0.1,
                   seed=9, sys_id=0, sched=O.SCHED_FL, direction=1, nsched=1000, trace_every=0)
    orc.run(nsteps)
    from paper_2103_10449_gb300 import nefe
    ctx = nefe.Context(precision=precision, skin=SKIN, nbr_cap=CAP)
    s = ctx.add_system(x0, box, v=v0, r0=x0)
    ctx.set_thermostat(s, T, 0.1, 9)
    ctx.set_schedule(s, nefe.NEFE_SCHED_FL, direction=1, nsteps=1000, k_E=5.0)
    if lanes is not None or gather_lanes is not None or list_lanes is not None:
        ctx.set_tuning(lanes if lanes is not None else 8, gather_lanes, list_lanes)
    ctx.run(nsteps)
    res = ctx.results(s)
    x, v, _ = ctx.get_state(s)
    ctx.close()
    return orc, res, x, v


def test_frenkel_ladd_trajectory_fp64_matches_oracle(N):
    orc, res, x, v = _fl_pair(1)
    ro = orc.results()
    assert res["step"] == ro["step"] == 300
    assert np.abs(x - orc.x).max() < 1e-8
    assert np.abs(v - orc.v).max() < 1e-6
    assert res["W"] == pytest.approx(ro["W"], rel=1e-8, abs=1e-9)
    assert res["lambda"] == pytest.approx(ro["lam"], rel=1e-14)
    assert res["U"] == pytest.approx(ro["U"], rel=1e-9)
    assert res["U_E"] == pytest.approx(ro["U_E"], rel=1e-7, abs=1e-9)
    assert res["T"] == pytest.approx(ro["T"], rel=1e-7)


@pytest.mark.parametrize("lanes", [0, 1, 4, 8, 16, 32])
def test_frenkel_ladd_trajectory_fp32_close_to_oracle(N, lanes):
    orc, res, x, v = _fl_pair(0, nsteps=100, lanes=lanes)
    ro = orc.results()
    # 100 FP32 steps of the 64-atom crystal stay within 3e-6 A and 1.3e-7 of W (measured on GB300)
    assert np.abs(x - orc.x).max() < 2e-5
    assert res["W"] == pytest.approx(ro["W"], rel=1e-6, abs=1e-9)
    assert res["U"] == pytest.approx(ro["U"], rel=1e-5)


@pytest.mark.parametrize("gather_lanes", [1, 2, 4, 8])
def test_pass_b_lanes_close_to_oracle(N, gather_lanes):
    orc, res, x, v = _fl_pair(0, nsteps=100, gather_lanes=gather_lanes)
    ro = orc.results()
    assert np.abs(x - orc.x).max() < 1e-4
    assert res["U"] == pytest.approx(ro["U"], rel=1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_list_forms_leave_the_run_bitwise_unchanged(N, precision):
    """The list build's output is integer and ranked by atom index: its form (one warp per
    cell, or 8, 16, 32 lanes per atom) cannot change anything downstream."""
    runs = [_fl_pair(precision, nsteps=150, list_lanes=ll) for ll in (0, 8, 16, 32)]
    for r in runs[1:]:
        assert r[1]["W"] == runs[0][1]["W"] and np.array_equal(r[2], runs[0][2])


@pytest.mark.parametrize("lanes", [None, 0])
def test_run_is_bitwise_deterministic(N, lanes):
    """Gather form (default lanes) and scatter form (integer accumulators): identical reruns."""
    a = _fl_pair(0, nsteps=200, lanes=lanes)
    b = _fl_pair(0, nsteps=200, lanes=lanes)
    assert a[1]["W"] == b[1]["W"] and np.array_equal(a[2], b[2])


def test_fused_epilogue_leaves_the_trajectory_bitwise_unchanged(N):
    """In the scatter form, every step of a sequence but the last runs the next step's kick,
    drift and noise inside its epilogue for the systems without a barostat.  101 steps in one
    call (three 32-step graphs with fused epilogues, then five steps) must equal, bit for bit,
    101 calls of one unfused step each -- for an NVT switching system (fused), an NPT system
    (never fused) and list rebuilds along the way."""
    from paper_2103_10449_gb300 import nefe
    x0, box = I.diamond(3, 3, 3)
    v0 = I.gaussian_velocities(len(x0), _sv(1000.0), 61)

    def make():
        ctx = nefe.Context(precision=nefe.NEFE_FP32, skin=SKIN, nbr_cap=CAP)
        a = ctx.add_system(x0, box, v=v0, r0=x0)
        ctx.set_thermostat(a, 1000.0, 0.1, 62)
        ctx.set_schedule(a, nefe.NEFE_SCHED_FL, nsteps=400, k_E=5.0)
        b = ctx.add_system(x0, box, v=v0)
        ctx.set_thermostat(b, 1000.0, 0.1, 63)
        ctx.set_barostat(b, nefe.NEFE_BARO_ISO, 1.0, 1.0)
        ctx.set_tuning(0)
        return ctx
    one, many = make(), make()
    one.run(101)
    for _ in range(101):
        many.run(1)
    for s in range(2):
        ra, rb = one.results(s), many.results(s)
        assert ra["step"] == rb["step"] == 101 and ra["error"] == rb["error"] == 0
        assert ra["W"] == rb["W"] and ra["U"] == rb["U"] and ra["T"] == rb["T"]
        xa, va, ba = one.get_state(s)
        xb, vb, bb = many.get_state(s)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ba, bb)
    builds = one.list_stats(0)[2]
    one.close()
    many.close()
    assert builds > 1


@pytest.mark.parametrize("lanes", [1, 0])
def test_thread_per_atom_pass_a_with_spilled_shells(N, lanes):
    """A random liquid has in-cutoff shells beyond the 8 entries the one-thread-per-atom pass A
    keeps in shared memory; the rest live in its global spill area.  Ten FP32 steps against the
    FP64 oracle (NVT, 1700 K)."""
    x0, box = I.liquid(512, 0.05425, seed=81)
    v0 = I.gaussian_velocities(len(x0), _sv(1700.0), 82)
    orc = O.System(x=x0.copy(), v=v0.copy(), box=box.copy(), T=1700.0, tdamp=0.1, seed=83, sys_id=0)
    orc.run(10)
    from paper_2103_10449_gb300 import nefe
    ctx = nefe.Context(precision=nefe.NEFE_FP32, skin=SKIN, nbr_cap=CAP)
    s = ctx.add_system(x0, box, v=v0)
    ctx.set_thermostat(s, 1700.0, 0.1, 83)
    ctx.set_tuning(lanes)
    ctx.run(10)
    _, mx = ctx.shell_stats()
    res = ctx.results(s)
    x, v, _ = ctx.get_state(s)
    ctx.close()
    assert mx > 8
    assert res["error"] == 0
    assert np.abs(x - orc.x).max() < 1e-4
    assert res["U"] == pytest.approx(orc.results()["U"], rel=1e-5)


def test_autotune_leaves_the_run_unchanged(N):
    """The autotuner's step-level timing runs on a snapshot that it restores: a run that
    autotunes midway equals, bit for bit, one that sets the chosen lanes and rebuild policy by
    hand."""
    from paper_2103_10449_gb300 import nefe
    x0, box = I.diamond(4, 4, 4)
    v0 = I.gaussian_velocities(len(x0), _sv(1000.0), 91)

    def make():
        ctx = nefe.Context(precision=nefe.NEFE_FP32, skin=SKIN, nbr_cap=CAP)
        for r in range(3):
            s = ctx.add_system(x0, box, v=v0, r0=x0)
            ctx.set_thermostat(s, 1000.0, 0.1, 92 + r)
            ctx.set_schedule(s, nefe.NEFE_SCHED_FL, nsteps=500, k_E=5.0)
        return ctx
    a = make()
    a.run(64)
    a.autotune()
    la = a.lanes()
    pol = a.rebuild_policy()
    a.run(64)
    ra = a.results_all()
    xa = [a.get_state(s)[0] for s in range(3)]
    a.close()
    b = make()
    b.run(64)
    b.set_tuning(la[0], la[1], la[2])
    b.set_rebuild_policy(pol)
    b.run(64)
    rb = b.results_all()
    xb = [b.get_state(s)[0] for s in range(3)]
    b.close()
    for s in range(3):
        assert ra[s]["step"] == rb[s]["step"] == 128
        assert ra[s]["W"] == rb[s]["W"]
        assert np.array_equal(xa[s], xb[s])

"""Parity at the benchmark's full size.

* The benchmark's own context (128 x 8000-atom Si-cd, Frenkel-Ladd at 1000 K, FP32 kernels, autotuned launch
  configuration, captured graph): after equilibration, autotuning and further steps, the SW energy and the
  Einstein spring energy the device reports for sampled replicas equal the oracle's energy of the state read
  back (1e-5 relative, the FP32 kernel tolerance).
* The stateless force path on one 1,000,000-atom rattled diamond cell, FP32 and FP64: forces on sampled atoms
  against the oracle's per-atom brute force (1e-5 / 1e-10 of the sampled force scale).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


def test_bench_configuration_energies_match_oracle(N):
    import bench
    stream = torch.cuda.Stream()
    ctx, n = bench.build_context(N, 128, N.NEFE_FP32, seed0=1000, stream=stream)
    ctx.run(96)
    ctx.autotune()
    ctx.run(64)
    ctx.sync()
    res = ctx.results_all()
    assert all(r["error"] == 0 for r in res)
    x0, _ = I.diamond(bench.NCELL, bench.NCELL, bench.NCELL)
    for s in (0, 37, 127):
        x, v, box = ctx.get_state(s)
        e_o = O.sw_energy(x, box)[0]
        assert res[s]["U"] == pytest.approx(e_o, rel=1e-5), s
        d = x - x0
        ue = 0.5 * bench.K_E * float(np.sum(d * d))
        assert res[s]["U_E"] == pytest.approx(ue, rel=1e-5, abs=1e-3), s
        assert res[s]["step"] == 160
    ctx.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-10)])
def test_million_atom_forces_sampled(N, precision, tol):
    x, box = I.diamond(50, 50, 50)
    x = I.rattle(x, 0.1, 71)
    n = len(x)
    assert n == 1_000_000
    cap = 48
    rcs = O.SW_SI[6] * O.SW_SI[1] + 0.5
    xd = torch.tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=torch.float64, device="cuda")
    nbr = torch.zeros(n * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    N.nefe_neighbor_build(xd, n, box, rcs, cap, nbr, cnt)
    f = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    N.nefe_sw_forces(xd, n, box, rcs, nbr, cnt, cap, N.params_from(O.SW_SI), precision, f)
    torch.cuda.synchronize()
    fg = f.cpu().numpy().reshape(3, n).T
    idx = np.random.default_rng(72).choice(n, 24, replace=False)
    f_o = O.sw_force_atoms(x, box, idx)
    assert np.abs(fg[idx] - f_o).max() <= tol * np.abs(f_o).max()


def _energies_match(N, ctx, systems):
    res = ctx.results_all()
    assert all(r["error"] == 0 for r in res)
    for s in systems:
        x, v, box = ctx.get_state(s)
        e_o = O.sw_energy(x, box)[0]
        assert res[s]["U"] == pytest.approx(e_o, rel=1e-5), s
    return res


def test_batched_dcci_configuration_energies_match_oracle(N):
    """The batched dCCI workload the bench times (64 Si-cd / beta-Sn pairs, 512..32768 atoms per
    phase, pressure control, barostats on; 1,008,516 atoms): after equilibration, autotuning and
    further steps, sampled systems' SW energies against the oracle's energy of the state read
    back, and every pair's lambda and scaled pressure finite and error-free."""
    import math
    import bench
    sizes = I.log_uniform_sizes(64, 512, 32768, seed=2021)
    sv = math.sqrt(O.KB * 400.0 / (O.M_SI * O.MVV2E))
    ctx = N.Context(precision=N.NEFE_FP32, dt=0.001, skin=bench.SKIN, nbr_cap=48)
    pids, natoms = [], []
    for k, n in enumerate(sizes):
        xa, ba = I.diamond(*I.diamond_cells_for(n))
        xb, bb = I.beta_tin(*I.beta_tin_cells_for(n))
        a = ctx.add_system(xa, ba, v=I.gaussian_velocities(len(xa), sv, 3000 + 2 * k))
        b = ctx.add_system(xb, bb, v=I.gaussian_velocities(len(xb), sv, 3001 + 2 * k))
        ctx.set_thermostat(a, 400.0, 0.1, 3000 + 2 * k)
        ctx.set_thermostat(b, 400.0, 0.1, 3001 + 2 * k)
        ctx.set_barostat(a, N.NEFE_BARO_ISO, 10.0, 0.5)
        ctx.set_barostat(b, N.NEFE_BARO_ANISO, 10.0, 0.5)
        pids.append(ctx.pair_dcci(a, b, 400.0, 10.0, N.NEFE_DCCI_PRESS, 10.0, 15.0, 100000))
        natoms += [len(xa), len(xb)]
    ctx.run(96)
    ctx.autotune()
    ctx.run(64)
    order = np.argsort(natoms)
    _energies_match(N, ctx, [int(order[0]), int(order[1]), int(order[len(order) // 2])])
    for p in pids:
        T_c, P_c, lam, err = ctx.pair(p)
        assert err == 0 and np.isfinite(lam) and np.isfinite(P_c)
    ctx.close()


def test_rs_npt_configuration_energies_match_oracle(N):
    """Reversible scaling NPT on the three phases of the bench's NPT workload (8000-atom Si-cd,
    8192-atom beta-Sn, 8000-atom liquid at 10 GPa; barostats move the boxes): sampled energies
    against the oracle after equilibration, autotuning and further steps."""
    import math
    import bench
    sv = math.sqrt(O.KB * 400.0 / (O.M_SI * O.MVV2E))
    ctx = N.Context(precision=N.NEFE_FP32, dt=0.001, skin=bench.SKIN, nbr_cap=48)
    phases = ((I.diamond(10, 10, 10), N.NEFE_BARO_ISO), (I.beta_tin(8, 16, 16), N.NEFE_BARO_ANISO),
              (I.liquid(8000, 0.05425, seed=4242), N.NEFE_BARO_ISO))
    for k, ((x, box), baro) in enumerate(phases):
        for r in range(4):
            s = ctx.add_system(x, box, v=I.gaussian_velocities(len(x), sv, 6100 + 4 * k + r))
            ctx.set_thermostat(s, 400.0, 0.1, 6100 + 4 * k + r)
            ctx.set_barostat(s, baro, 10.0, 1.0)
            ctx.set_schedule(s, N.NEFE_SCHED_RS, nsteps=50000, lambda_f=0.2, P_GPa=10.0)
    ctx.run(96)
    ctx.autotune()
    ctx.run(64)
    res = _energies_match(N, ctx, [0, 5, 10])
    for k, ((x, box), _) in enumerate(phases):
        assert not np.allclose(res[4 * k]["box"], box)      # the barostat moved every box
    ctx.close()

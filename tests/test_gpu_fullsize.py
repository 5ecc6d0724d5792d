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

"""Pins of the FP64 oracle against what the physics and mathematics fix (no GPU).

Every check here compares the oracle with something other than itself: a library routine
(numpy's Philox, scipy's KD-tree and normal distribution, numpy's lexsort), a closed form
(Einstein crystal, harmonic switching, reversible scaling of a harmonic crystal), a
published property of the Stillinger-Weber parametrisation (pair minimum -eps at
2^(1/6) sigma; diamond cohesive energy -2 eps), finite differences, invariances, or an
algebraic identity between two of the paper's equations.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


def _sv(T):
    return math.sqrt(O.KB * T / (O.M_SI * O.MVV2E))


# ---------------------------------------------------------------- Philox / thermostat noise
@pytest.mark.parametrize("ctr,key", [((0, 0, 0, 0), (0, 0)), ((7, 8, 9, 10), (123, 456)),
                                     ((2**64 - 2, 2**63, 5, 2**40), (2**64 - 1, 99))])
def test_philox_matches_numpy(ctr, key):
    # numpy's Philox (4x64, 10 rounds) pre-increments its 256-bit counter (word 0 lowest)
    # before each block, so it is seeded with ctr - 1.
    c = (sum(w << (64 * i) for i, w in enumerate(ctr)) - 1) % 2**256
    before = [(c >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(before, dtype=np.uint64))
    ref = bg.random_raw(4)
    got = O.philox4x64(ctr, key)
    assert np.array_equal(ref, got)


def test_langevin_noise_is_standard_normal():
    from scipy import stats
    xi = O.langevin_xi(seed=11, sys_id=3, step=17, n=100000)
    z = xi.ravel()
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    c = np.corrcoef(xi.T)
    assert np.abs(c - np.eye(3)).max() < 5.0 / math.sqrt(xi.shape[0])
    # counter-based: another step or system gives an independent stream, same step repeats
    assert np.array_equal(xi, O.langevin_xi(11, 3, 17, 100000))
    assert abs(np.corrcoef(xi[:, 0], O.langevin_xi(11, 3, 18, 100000)[:, 0])[0, 1]) < 0.02


# ---------------------------------------------------------------- Stillinger-Weber energy
def test_sw_cohesive_energy_diamond():
    g = _golden("sw_si.txt")
    x, box = I.diamond(2, 2, 2, a=5.431)
    e, f, vir, ea = O.sw_energy(x, box)
    assert abs(e / len(x) - g["cohesive_energy_a5431"]) < 1e-6
    assert np.abs(f).max() < 1e-12
    # at the lattice constant where r_nn = 2^(1/6) sigma the energy is exactly -2 eps
    eps, sig = O.SW_SI[0], O.SW_SI[1]
    a0 = 4.0 * 2.0 ** (1.0 / 6.0) * sig / math.sqrt(3.0)
    x, box = I.diamond(3, 3, 3, a=a0)
    e, _, _, _ = O.sw_energy(x, box)
    assert abs(e / len(x) + 2.0 * eps) < 1e-9 * eps      # A, B are published to 10 digits


def _dimer(r):
    x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    return O.sw_energy(x, np.array([20.0, 20.0, 20.0]))


def test_sw_pair_minimum_is_minus_eps_at_two_sixth_sigma():
    eps, sig, a = O.SW_SI[0], O.SW_SI[1], O.SW_SI[6]
    r0 = 2.0 ** (1.0 / 6.0) * sig
    e0, f0, _, _ = _dimer(r0)
    assert abs(e0 + eps) < 1e-9
    assert np.abs(f0).max() < 1e-6
    for dr in (-0.05, 0.05, 0.3):
        assert _dimer(r0 + dr)[0] > e0
    # smooth cutoff at a sigma
    assert _dimer(a * sig - 1e-9)[0] == pytest.approx(0.0, abs=1e-12)
    assert _dimer(a * sig + 1e-3)[0] == 0.0


def test_three_body_vanishes_at_tetrahedral_angle():
    # Diamond only has tetrahedral bonds inside a sigma: E/N = 2 phi2(r_nn) for any a.
    for a in (5.35, 5.431, 5.55):
        x, box = I.diamond(2, 2, 2, a=a)
        e, _, _, _ = O.sw_energy(x, box)
        e_pair = _dimer(a * math.sqrt(3.0) / 4.0)[0]
        assert e / len(x) == pytest.approx(2.0 * e_pair, rel=1e-12, abs=1e-12)


def _trimer(r, theta):
    c = np.array([10.0, 10.0, 10.0])
    x = np.array([c, c + [r, 0, 0], c + [r * math.cos(theta), r * math.sin(theta), 0.0]])
    return O.sw_energy(x, np.array([30.0, 30.0, 30.0]))[0]


def test_three_body_angular_and_radial_dependence():
    eps, sig, lam, gam, a, c0 = (O.SW_SI[0], O.SW_SI[1], O.SW_SI[7], O.SW_SI[8],
                                 O.SW_SI[6], O.SW_SI[9])
    r = 2.3
    e2 = _dimer(r)[0]
    # right angle: the two legs' far ends are r*sqrt(2) = 3.25 A apart (inside a sigma)
    e_lin = _trimer(r, math.pi) - 2 * e2                  # one triplet, cos = -1
    e_rt = _trimer(r, math.pi / 2) - 2 * e2 - _dimer(r * math.sqrt(2))[0]
    e_eq = _trimer(r, math.pi / 3) - 3 * e2               # three triplets, cos = 1/2
    # two legs of length r at the centre; third-atom triplets involve the long r*sqrt(2) leg
    g = math.exp(gam * sig / (r - a * sig))
    gl = math.exp(gam * sig / (r * math.sqrt(2) - a * sig))
    assert e_lin == pytest.approx(eps * lam * (-1 - c0) ** 2 * g * g, rel=1e-12)
    assert e_eq / e_lin == pytest.approx(3 * (0.5 - c0) ** 2 / (-1 - c0) ** 2, rel=1e-12)
    # right triangle: centre angle 90 deg, two 45 deg angles with one long leg each
    expect_rt = eps * lam * ((0 - c0) ** 2 * g * g + 2 * (math.sqrt(0.5) - c0) ** 2 * g * gl)
    assert e_rt == pytest.approx(expect_rt, rel=1e-12)


def _fd_forces(x, box, h=1e-5):
    fd = np.zeros_like(x)
    for i in range(len(x)):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd[i, k] = -(O.sw_energy(xp, box)[0] - O.sw_energy(xm, box)[0]) / (2 * h)
    return fd


@pytest.mark.parametrize("kind", ["diamond", "beta_tin", "liquid"])
def test_forces_are_minus_gradient(kind):
    if kind == "diamond":
        x, box = I.diamond(2, 2, 2)
        x = I.rattle(x, 0.15, 5)
    elif kind == "beta_tin":
        x, box = I.beta_tin(2, 2, 4)
        x = I.rattle(x, 0.1, 6)
    else:
        x, box = I.liquid(48, 0.05425, seed=7, rmin=1.9)
    e, f, vir, ea = O.sw_energy(x, box)
    fd = _fd_forces(x, box)
    assert np.abs(fd - f).max() < 1e-6 * max(1.0, np.abs(f).max())
    assert np.abs(f.sum(axis=0)).max() < 1e-11
    assert ea.sum() == pytest.approx(e, rel=1e-13, abs=1e-12)
    sub = np.array([0, 3, len(x) - 1])
    assert np.abs(O.sw_force_atoms(x, box, sub) - f[sub]).max() < 1e-12


def test_virial_is_strain_derivative():
    x, box = I.beta_tin(2, 2, 4)
    x = I.rattle(x, 0.1, 8)
    e, f, vir, _ = O.sw_energy(x, box)
    h = 1e-6
    for a in range(3):   # W_aa = -dE/d(eps_aa) for x_a -> (1+eps) x_a, L_a -> (1+eps) L_a
        s = np.ones(3); s[a] += h
        ep = O.sw_energy(x * s, box * s)[0]
        s = np.ones(3); s[a] -= h
        em = O.sw_energy(x * s, box * s)[0]
        assert vir[a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-6)
    # Off-diagonal part on an isolated cluster (no bond crosses the boundary), where the
    # virial is sum_i x_i (x) f_i and d E / d(shear x += eps y) = -sum_i f_ix y_i.
    xl, bl = I.liquid(200, 0.05425, seed=12)
    c = xl[np.argsort(np.sum((xl - bl / 2) ** 2, axis=1))[:30]]
    c = c - c.mean(axis=0) + 20.0
    bigbox = np.array([40.0, 40.0, 40.0])
    _, _, vc, _ = O.sw_energy(c, bigbox)

    def e_shear(eps, a, b):
        y = c.copy(); y[:, a] += eps * (c[:, b] - 20.0)
        return O.sw_energy(y, bigbox)[0]
    for comp, (a, b) in ((3, (0, 1)), (4, (0, 2)), (5, (1, 2))):
        dab = (e_shear(h, a, b) - e_shear(-h, a, b)) / (2 * h)
        dba = (e_shear(h, b, a) - e_shear(-h, b, a)) / (2 * h)
        assert vc[comp] == pytest.approx(-0.5 * (dab + dba), rel=1e-6, abs=1e-6)


def test_invariances():
    x, box = I.liquid(60, 0.05425, seed=9, rmin=1.9)
    e, f, vir, ea = O.sw_energy(x, box)
    e2, f2, _, _ = O.sw_energy(x + np.array([1.3, -7.1, 40.2]), box)       # translation
    assert e2 == pytest.approx(e, rel=1e-12)
    assert np.abs(f2 - f).max() < 1e-10
    p = np.random.default_rng(0).permutation(len(x))                       # permutation
    e3, f3, _, _ = O.sw_energy(x[p], box)
    assert e3 == pytest.approx(e, rel=1e-12)
    assert np.abs(f3 - f[p]).max() < 1e-10
    xr = x[:, [1, 2, 0]]                                                     # axis rotation
    e4, f4, vir4, _ = O.sw_energy(xr, box[[1, 2, 0]])
    assert e4 == pytest.approx(e, rel=1e-12)
    assert np.abs(f4 - f[:, [1, 2, 0]]).max() < 1e-10
    assert np.allclose(vir4[:3], vir[[1, 2, 0]], rtol=1e-10, atol=1e-10)


# ---------------------------------------------------------------- neighbour list and cells
@pytest.mark.parametrize("kind", ["diamond64", "liquid", "beta_tin"])
def test_neighbor_list_matches_kdtree(kind):
    from scipy.spatial import cKDTree
    if kind == "diamond64":
        x, box = I.diamond(2, 2, 2); x = I.rattle(x, 0.2, 1)
    elif kind == "liquid":
        x, box = I.liquid(400, 0.05425, seed=2)
    else:
        x, box = I.beta_tin(4, 4, 8); x = I.rattle(x, 0.1, 3)
    rcs = 3.7712 + 0.5
    nbr, cnt, img = O.neighbor_list(x, box, rcs)
    xw = x - box * np.floor(x / box)
    pairs = cKDTree(xw, boxsize=box).query_pairs(rcs)
    ref = set()
    for i, j in pairs:
        ref.add((i, j)); ref.add((j, i))
    got = {(i, int(nbr[i, s])) for i in range(len(x)) for s in range(cnt[i])}
    assert got == ref
    for i in range(len(x)):                       # rows sorted by j; image reproduces distance
        row = nbr[i, :cnt[i]]
        assert np.all(np.diff(row) > 0)
        d = x[row] - x[i] - img[i, :cnt[i]] * box
        assert np.all(np.sum(d * d, axis=1) < rcs * rcs)


def test_cell_bin_is_stable_sort_by_cell():
    x, box = I.liquid(500, 0.05425, seed=4)
    x = x + np.array([100.0, -55.0, 3.0]) * box / box.max()     # unwrapped coordinates
    rcs = 4.2712
    nc3, cell_of, start, perm = O.cell_bin(x, box, rcs)
    assert np.all(box / nc3 >= rcs) and np.all(nc3 == np.floor(box / rcs))
    w = (x / box) - np.floor(x / box)
    c3 = np.minimum((w * nc3).astype(int), nc3 - 1)
    assert np.array_equal(cell_of, c3[:, 0] + nc3[0] * (c3[:, 1] + nc3[1] * c3[:, 2]))
    assert np.array_equal(perm, np.lexsort((np.arange(len(x)), cell_of)))
    assert np.array_equal(start, np.searchsorted(np.sort(cell_of), np.arange(nc3.prod() + 1)))


# ---------------------------------------------------------------- closed forms
def test_einstein_free_energy_closed_form():
    g = _golden("einstein.txt")
    assert O.einstein_free_energy(1, 5.0, 400.0) == pytest.approx(g["k5_T400"], abs=5e-7)
    assert O.einstein_free_energy(1, 5.0, 1000.0) == pytest.approx(g["k5_T1000"], abs=5e-7)
    assert O.einstein_free_energy(1, 6.113, 400.0) == pytest.approx(g["k6.113_T400"], abs=5e-7)
    assert O.einstein_free_energy(1, 1.362, 400.0) == pytest.approx(g["k1.362_T400"], abs=5e-7)
    # classical limit of the quantum oscillator, 3 kT ln(1 - exp(-x)) + 3 hw/2 -> 3 kT ln x
    k, T = 5.0, 1e6
    w = math.sqrt(k / (O.M_SI * O.MVV2E))
    xq = O.HBAR * w / (O.KB * T)
    fq = 3 * (0.5 * O.HBAR * w + O.KB * T * math.log(-math.expm1(-xq)))
    assert O.einstein_free_energy(1, k, T) == pytest.approx(fq, rel=1e-6)


def test_fl_schedule_shape():
    tau = np.linspace(0, 1, 2001)
    lam = O.fl_lambda(tau)
    assert lam[0] == 0.0 and lam[-1] == pytest.approx(1.0, abs=1e-14)
    assert np.all(np.diff(lam) >= 0)
    assert np.allclose(O.fl_lambda(1 - tau), 1 - lam, atol=1e-12)      # odd about 1/2
    d = np.gradient(lam, tau)
    assert abs(d[0]) < 1e-6 and abs(d[-1]) < 1e-6


def test_rs_schedule_temperature_is_linear():
    tau = np.linspace(0, 1, 11)
    lam = O.rs_lambda(tau, 400.0 / 2000.0)
    T = 400.0 / lam
    assert np.allclose(np.diff(T), 160.0)


def test_dcci_press_update_is_temp_update_rearranged():
    rng = np.random.default_rng(5)
    for _ in range(100):
        lam_k, p_k, p_k1 = rng.uniform(0.3, 1.5), rng.uniform(-0.05, 0.1), rng.uniform(-0.05, 0.1)
        du, dv = rng.uniform(-0.3, 0.3), rng.uniform(-3.0, 3.0)
        lam_k1 = O.dcci_press_update(lam_k, p_k, p_k1, du, dv)
        # Eq. l_coex_discreted must satisfy Eq. Ps_coex_discreted with P_S = lambda P
        ps_k1 = O.dcci_temp_update(lam_k * p_k, lam_k, lam_k1, du, dv)
        assert ps_k1 == pytest.approx(lam_k1 * p_k1, rel=1e-10, abs=1e-13)


def test_estimators():
    assert O.free_energy_difference([3.0, 5.0], [-1.0, -3.0]) == 3.0
    assert O.dissipated_heat([3.0, 5.0], [-1.0, -3.0]) == 1.0
    assert O.gibbs_from_helmholtz(-4.0, 0.01, 20.0) == pytest.approx(-3.8)
    assert O.gibbs_rs(-4.0, 1, 400.0, 1.0, 0.0, 0.0) == pytest.approx(-4.0)


# ---------------------------------------------------------------- integrator and thermostat
def _diamond_system(temp=400.0, vseed=1, **kw):
    x, box = I.diamond(2, 2, 2)
    v = I.gaussian_velocities(len(x), _sv(temp), vseed)
    return O.System(x=x.copy(), v=v, box=box.copy(), **kw)


def test_nve_energy_conservation_and_reversibility():
    s = _diamond_system()
    s.setup()
    e0 = s.u_int + 0.5 * s.kt[:3].sum()
    es = []
    for _ in range(1000):
        s.step()
        es.append(s.u_int + 0.5 * s.kt[:3].sum())
    es = np.array(es)
    assert abs(es[-1] - e0) / s.n < 2e-4 and (es.max() - es.min()) / s.n < 3e-4
    x0, v0 = s.x.copy(), s.v.copy()
    s.run(200)
    s.v = -s.v
    s.run(200)
    assert np.abs(s.x - x0).max() < 1e-9 and np.abs(s.v + v0).max() < 1e-7


def _harmonic(k_a, k_b, T, direction, seed, nsw=2000, neq=1000):
    """Equilibrate at the starting end state, then switch k_a (lambda=0) <-> k_b (lambda=1)."""
    x, box = I.diamond(2, 2, 2)
    v = I.gaussian_velocities(len(x), _sv(T), seed)
    k_start = k_a if direction > 0 else k_b
    eq = O.System(x=x.copy(), v=v, box=box.copy(), pot=O.POT_EINSTEIN, k_int=k_start,
                  r0=x.copy(), T=T, tdamp=0.1, seed=seed, sys_id=1)
    eq.run(neq)
    sw = O.System(x=eq.x, v=eq.v, box=box.copy(), pot=O.POT_EINSTEIN, k_int=k_a, r0=x.copy(),
                  k_E=k_b, T=T, tdamp=0.1, seed=seed, sys_id=2, sched=O.SCHED_FL,
                  direction=direction, nsched=nsw)
    sw.run(nsw)
    return sw.W


def test_harmonic_switching_reproduces_closed_form():
    T, n = 400.0, 64
    wf = [_harmonic(5.0, 10.0, T, +1, s) for s in range(4)]
    wb = [_harmonic(5.0, 10.0, T, -1, 100 + s) for s in range(4)]
    dF = O.free_energy_difference(wf, wb) / n
    exact = 1.5 * O.KB * T * math.log(10.0 / 5.0)
    assert abs(dF - exact) < 1e-3                          # 1 meV/atom
    assert 0.0 < O.dissipated_heat(wf, wb) / n < 5e-3      # second law: dissipation >= 0
    # Eq. dA: the system at lambda = 0 (spring 5) from the reference at lambda = 1 (spring 10).
    # A sign error (F_ref + dF) would miss the closed form by 2 dF = 72 meV/atom.
    f_int = O.helmholtz_from_switching(O.einstein_free_energy(n, 10.0, T), wf, wb)
    assert abs(f_int - O.einstein_free_energy(n, 5.0, T)) / n < 1e-3


def test_langevin_equipartition_harmonic():
    T = 400.0
    s = _diamond_system(temp=T, vseed=3, pot=O.POT_EINSTEIN, k_int=5.0, T=T, tdamp=0.1, seed=3)
    s.r0 = s.x.copy()
    s.run(500)
    K, U = [], []
    for _ in range(4000):
        s.step()
        K.append(0.5 * s.kt[:3].sum()); U.append(s.u_int)
    n = s.n
    assert np.mean(K) / ((3 * n - 3) / 2 * O.KB * T) == pytest.approx(1.0, abs=0.05)
    assert np.mean(U) / (1.5 * n * O.KB * T) == pytest.approx(1.0, abs=0.05)
    assert np.abs(s.v.sum(axis=0)).max() < 1e-8           # net random force removed


def test_reversible_scaling_of_einstein_crystal():
    """RS with U_int an Einstein crystal: Eq. Gibbs_RS must give F(k, T0/lambda) exactly."""
    T0, k, lam_f, n = 400.0, 5.0, 0.5, 64
    nsw = 2000

    def run(direction, seed):
        x, box = I.diamond(2, 2, 2)
        v = I.gaussian_velocities(len(x), _sv(T0), seed)
        k_eq = k if direction > 0 else lam_f * k
        eq = O.System(x=x.copy(), v=v, box=box.copy(), pot=O.POT_EINSTEIN, k_int=k_eq,
                      r0=x.copy(), T=T0, tdamp=0.1, seed=seed, sys_id=1)
        eq.run(1000)
        rs = O.System(x=eq.x, v=eq.v, box=box.copy(), pot=O.POT_EINSTEIN, k_int=k, r0=x.copy(),
                      T=T0, tdamp=0.1, seed=seed, sys_id=2, sched=O.SCHED_RS, direction=direction,
                      nsched=nsw, lam_f=lam_f, p_ext=0.0)
        rs.run(nsw)
        return rs.W
    wf = [run(+1, s) for s in range(4)]
    wb = [run(-1, 50 + s) for s in range(4)]
    g0 = O.einstein_free_energy(n, k, T0)
    g = O.gibbs_rs(g0, n, T0, lam_f, np.mean(wf), np.mean(wb))
    exact = O.einstein_free_energy(n, k, T0 / lam_f)
    assert abs(g - exact) / n < 1e-3


def test_barostat_restores_target_pressure():
    """Parrinello-Rahman-type iso box equation: a compressed crystal expands; the mean
    pressure over a run settles at the target (an invariant, not a value from the paper)."""
    T = 400.0
    s = _diamond_system(temp=T, vseed=4, T=T, tdamp=0.1, baro=O.BARO_ISO, p_ext=0.0, pdamp=0.5)
    s.x *= 0.99
    s.box *= 0.99
    v0 = s.volume()
    s.run(200)
    assert s.volume() > v0
    s.run(1000)
    P = []
    for _ in range(3000):
        s.step()
        P.append(s.observe()[2])
    assert abs(np.mean(P)) * O.EV_A3_TO_GPA < 0.3         # GPa, fluctuations ~1 GPa at 64 atoms


def _ideal_gas_as_work(n, seed, p_from, p_to, nsched, n_eq, T, baro=O.BARO_ISO, shape=(1.0, 1.0, 1.0)):
    """Work of one pressure switch p_from -> p_to of n non-interacting atoms (U = 0) after
    n_eq steps of NPT equilibration at p_from; pressures in eV/A^3.  ``shape`` gives the box
    edge ratios (a tetragonal box for the anisotropic box equation)."""
    kT = O.KB * T
    L = ((n - 1) * kT / p_from / np.prod(shape)) ** (1.0 / 3.0)
    box = L * np.asarray(shape, dtype=np.float64)
    x = np.random.default_rng(seed).uniform(0.0, 1.0, (n, 3)) * box
    common = dict(pot=O.POT_EINSTEIN, k_int=0.0, T=T, tdamp=0.1, sys_id=0, baro=baro, p_ext=p_from,
                  pdamp=0.5)
    eq = O.System(x=x, v=I.gaussian_velocities(n, _sv(T), seed), box=box, r0=x.copy(), seed=seed,
                  **common)
    eq.run(n_eq)
    sw = O.System(x=eq.x.copy(), v=eq.v.copy(), box=eq.box.copy(), r0=eq.x.copy(), seed=seed + 1000,
                  sched=O.SCHED_AS, nsched=nsched, p0=p_from, p1=p_to, **common)
    sw.eta = eq.eta.copy()
    sw.run(nsched)
    return sw.W


@pytest.mark.parametrize("baro,shape", [(O.BARO_ISO, (1.0, 1.0, 1.0)), (O.BARO_ANISO, (1.0, 1.0, 0.6))])
def test_pressure_switching_of_an_ideal_gas_closed_form(baro, shape):
    """Adiabatic switching in pressure (Sec. 2.3, Eq. Gibbs_AS) of an ideal gas, 16 atoms at
    400 K, 0.1 -> 0.3 GPa and back, 8 + 8 realisations of 10 ps.  With U = 0 the virial vanishes,
    so P_inst V = 2K/3.  The box equation is stationary only if <V (P_inst - P)> = 0, and the
    thermostat, which removes the net momentum, leaves 3N - 3 degrees of freedom: <2K/3> =
    (N - 1) kB T.  Hence <V>(P) = (N - 1) kB T / P and the reversible work is
    dG = (N - 1) kB T ln(P1 / P0), the ideal gas's Gibbs energy change with N - 1 for N.
    This pins the switching work (left-point sum of V dP, pressure units, sign), the estimator
    and the barostat's mechanical equilibrium; a 3N-degree count would be off by 1/16 = 6 %.
    The anisotropic box equation (one strain rate per axis, driven by P_aa) runs the same
    switch in a tetragonal box: each axis is stationary only at <V (P_aa - P)> = 0, and for
    the ideal gas every P_aa V is 2 K_a with K_a the kinetic energy of that axis (N - 1 degrees
    of freedom each), which gives the same closed form."""
    n, T = 16, 400.0
    p0, p1 = 0.1 / O.EV_A3_TO_GPA, 0.3 / O.EV_A3_TO_GPA
    reps, nsched, n_eq = 8, 10000, 2000
    wf = np.array([_ideal_gas_as_work(n, 10 + r, p0, p1, nsched, n_eq, T, baro, shape) for r in range(reps)])
    wb = np.array([_ideal_gas_as_work(n, 40 + r, p1, p0, nsched, n_eq, T, baro, shape) for r in range(reps)])
    dG = float(O.gibbs_as(0.0, wf.mean(), wb.mean()))
    exact = (n - 1) * O.KB * T * math.log(p1 / p0)
    sem = 0.5 * math.sqrt(wf.var(ddof=1) / reps + wb.var(ddof=1) / reps)
    assert sem < 0.01 * exact
    assert abs(dG / exact - 1.0) < 0.03          # about four standard errors


def _ideal_gas_rs_work(n, seed, P, lam_f, direction, nsched, n_eq, T):
    """Work of one reversible-scaling switch (NPT, physical pressure P in eV/A^3) of n
    non-interacting atoms, after n_eq steps of equilibration at the starting lambda (1
    forward, lam_f backward), where the barostat target is lambda P."""
    kT = O.KB * T
    lam0 = 1.0 if direction > 0 else lam_f
    L = ((n - 1) * kT / (lam0 * P)) ** (1.0 / 3.0)
    x = np.random.default_rng(seed).uniform(0.0, L, (n, 3))
    common = dict(pot=O.POT_EINSTEIN, k_int=0.0, T=T, tdamp=0.1, sys_id=0, baro=O.BARO_ISO, pdamp=0.5)
    eq = O.System(x=x, v=I.gaussian_velocities(n, _sv(T), seed), box=np.array([L, L, L]), r0=x.copy(), seed=seed,
                  p_ext=lam0 * P, **common)
    eq.run(n_eq)
    sw = O.System(x=eq.x.copy(), v=eq.v.copy(), box=eq.box.copy(), r0=eq.x.copy(), seed=seed + 1000, p_ext=P,
                  sched=O.SCHED_RS, direction=direction, nsched=nsched, lam_f=lam_f, **common)
    sw.eta = eq.eta.copy()
    sw.run(nsched)
    return sw.W


def test_reversible_scaling_npt_of_an_ideal_gas_closed_form():
    """Reversible scaling at constant pressure (Sec. 2.2, Eq. dH_RS with P_S = lambda P, the
    barostat target of the ``ners`` tag) of an ideal gas, 16 atoms, T0 = 400 K, P = 0.1 GPa,
    lambda 1 -> 0.5 and back, 8 + 8 realisations of 10 ps.  With U = 0 the driving force is
    P V, and at target lambda P the box settles at <V> = (N - 1) kB T0 / (lambda P) (as in the
    pressure-switching pin), so the reversible work is the integral of (N - 1) kB T0 / lambda,
    i.e. (N - 1) kB T0 ln(lambda_f).  Together with the kinetic term of Eq. Gibbs_RS this is the
    ideal gas's G(T) = (T/T0) G(T0) - 5/2 N kB T ln(T/T0), up to the N - 1 degrees count."""
    n, T0, P, lam_f = 16, 400.0, 0.1 / O.EV_A3_TO_GPA, 0.5
    reps, nsched, n_eq = 8, 10000, 2000
    wf = np.array([_ideal_gas_rs_work(n, 10 + r, P, lam_f, 1, nsched, n_eq, T0) for r in range(reps)])
    wb = np.array([_ideal_gas_rs_work(n, 40 + r, P, lam_f, -1, nsched, n_eq, T0) for r in range(reps)])
    w_rev = 0.5 * (wf.mean() - wb.mean())
    exact = (n - 1) * O.KB * T0 * math.log(lam_f)
    sem = 0.5 * math.sqrt(wf.var(ddof=1) / reps + wb.var(ddof=1) / reps)
    assert sem < 0.01 * abs(exact)
    assert abs(w_rev / exact - 1.0) < 0.03        # about four standard errors


def test_dcci_pair_replays_the_discrete_equations():
    """The pair update uses the instantaneous per-atom dU, dV of both systems each step and
    is the composition of Eq. Ps_coex_discreted / Eq. l_coex_discreted step by step."""
    a = _diamond_system(temp=400.0, vseed=5, T=400.0, tdamp=0.1, seed=5, sys_id=0, baro=O.BARO_ISO, pdamp=0.5)
    xb, bb = I.beta_tin(2, 2, 4)
    b = O.System(x=xb, v=I.gaussian_velocities(len(xb), _sv(400.0), 6), box=bb, T=400.0, tdamp=0.1,
                 seed=5, sys_id=1, baro=O.BARO_ANISO, pdamp=0.5)
    p0 = 10.0 / O.EV_A3_TO_GPA
    for mode, frm, to in ((O.DCCI_TEMP, 400.0, 500.0), (O.DCCI_PRESS, p0, p0 * 1.2)):
        pair = O.DcciPair(a, b, 400.0, p0, mode, frm, to, 50)
        pair.run(20)
        lam, ps = 1.0, p0
        for k, lam_k, ps_k, du, dv in pair.hist:
            assert lam_k == lam and ps_k == ps
            if mode == O.DCCI_TEMP:
                lam = frm / (frm + (to - frm) * (k + 1) / 50)
                ps = O.dcci_temp_update(ps, lam_k, lam, du, dv)
            else:
                pk, pk1 = frm + (to - frm) * k / 50, frm + (to - frm) * (k + 1) / 50
                lam = O.dcci_press_update(lam_k, pk, pk1, du, dv)
                ps = lam * pk1
        assert pair.error == 0
        T_c, P_c = pair.coexistence()
        assert T_c == pytest.approx(400.0 / pair.lam) and P_c == pytest.approx(pair.ps / pair.lam)


def test_anisotropic_box_equation_relaxes_each_axis_to_the_enthalpy_minimum():
    """The anisotropic box equation (the beta-Sn barostat of Sec. 4, ``nph aniso``) drives
    each axis by its own P_aa.  A 64-atom beta-Sn cell (A5 has no internal coordinate) started
    at c/a = 0.55 and run at 300 K and 10 GPa must relax to the lattice constants that minimise the
    static enthalpy E(a, b, c) + P a b c (found here by scipy over all three edges, thermal
    expansion at 300 K is below 1 %), and every diagonal pressure component must average to
    the target separately.  Driving all axes by the mean pressure would keep c/a at 0.55,
    4 % from the minimum, with P_zz and P_xx apart by several GPa."""
    from scipy.optimize import minimize
    P, T = 10.0 / O.EV_A3_TO_GPA, 300.0
    x1, b1 = I.beta_tin(2, 2, 4, a=1.0, c_over_a=1.0)

    def enthalpy(edges):
        e = O.sw_energy(x1 * (np.asarray(edges) / b1), np.asarray(edges))[0]
        return e + P * float(np.prod(edges))
    x0, box0 = I.beta_tin(2, 2, 4)
    opt = minimize(enthalpy, box0, method="Nelder-Mead", options=dict(xatol=1e-8, fatol=1e-12, maxiter=4000))
    s = O.System(x=x0.copy(), v=I.gaussian_velocities(len(x0), _sv(T), 3), box=box0.copy(), T=T, tdamp=0.1,
                 seed=3, baro=O.BARO_ANISO, p_ext=P, pdamp=0.5)
    s.run(3000)
    B, VP, V = [], [], []
    for k in range(6000):
        s.step()
        if k % 5 == 0:
            Vk, Pt = s.observe()[:2]
            B.append(s.box.copy())
            VP.append(Vk * Pt[:3])
            V.append(Vk)
    box = np.mean(B, axis=0)
    assert np.abs(box / opt.x - 1.0).max() < 0.01
    assert abs((box[2] / box[0]) / (opt.x[2] / opt.x[0]) - 1.0) < 0.01
    p_axes = np.mean(VP, axis=0) / np.mean(V) * O.EV_A3_TO_GPA
    assert np.abs(p_axes - 10.0).max() < 0.1                     # GPa, each axis separately


@pytest.mark.parametrize("baro,omega_tau", [(O.BARO_ISO, 3.0), (O.BARO_ANISO, math.sqrt(3.0))])
def test_box_equation_small_oscillation_frequency(baro, omega_tau):
    """Dynamics of the box equation (the reading: eta' = d V (P - P_target) / Q_b with
    Q_b = (N + 1) kB T tau_P^2, d = 3 for the isotropic form, d = 1 per axis for the anisotropic
    one, and ln V' = 3 eta resp. sum of the axes' eta).  For an ideal gas held at T by the
    thermostat, P V = (N - 1) kB T, so u = ln(V / V_eq) obeys u'' = -c (e^u - 1) with
    c = 9 (N - 1) kB T / Q_b (isotropic) or 3 (N - 1) kB T / Q_b (anisotropic: the three axes
    see the same kinetic pressure on average): small oscillations of the volume at
    omega tau_P = 3 resp. sqrt(3) (times sqrt((N - 1)/(N + 1))).  An isotropic factor d = 3
    on each axis of the anisotropic form, or a missing one in the isotropic form, changes
    omega by sqrt(3)."""
    n, T, P, tau_p = 4096, 400.0, 0.1 / O.EV_A3_TO_GPA, 0.5
    kT = O.KB * T
    v_eq = (n - 1) * kT / P
    L = (1.1 * v_eq) ** (1.0 / 3.0)
    box = np.array([L, L * 1.1, L / 1.1])
    x = np.random.default_rng(1).uniform(0.0, 1.0, (n, 3)) * box
    s = O.System(x=x, v=I.gaussian_velocities(n, _sv(T), 2), box=box, r0=x.copy(), pot=O.POT_EINSTEIN, k_int=0.0,
                 T=T, tdamp=0.1, seed=4, baro=baro, p_ext=P, pdamp=tau_p)
    s.setup()
    u = []
    for _ in range(4000):
        s.step()
        u.append(math.log(s.volume() / v_eq))
    u = np.array(u)
    cross = np.where(np.sign(u[:-1]) != np.sign(u[1:]))[0]
    assert len(cross) >= 4
    omega = math.pi / (np.diff(cross[:4]).mean() * s.dt)
    expect = omega_tau / tau_p * math.sqrt((n - 1) / (n + 1))
    assert abs(omega / expect - 1.0) < 0.1


class _FrozenPhase:
    """A phase whose per-atom energy and volume stay fixed: what the dCCI update sees when the
    two phases' dU and dV do not change along the line."""

    def __init__(self, n, u_atom, v_atom):
        self.n, self.u_int, self.vol = n, n * u_atom, n * v_atom
        self.f = np.zeros((n, 3))

    def setup(self):
        pass

    def observe(self):
        return self.vol, np.zeros(6), 0.0, 0.0, 0.0

    def record(self, *a):
        pass

    def barostat_kick(self, Pt):
        pass

    def particle_step(self):
        pass


@pytest.mark.parametrize("mode", [O.DCCI_TEMP, O.DCCI_PRESS])
def test_dcci_with_constant_latent_heat_follows_the_exact_clausius_clapeyron_line(mode):
    """With dU and dV per atom constant along the line, the Clausius-Clapeyron equation
    (Eq. CCE, dP/dT = (dU + P dV) / (T dV) per atom) integrates exactly to
    P/T = P0/T0 - (dU/dV)(1/T - 1/T0).  The discrete updates (Eqs. Ps_coex_discreted and
    l_coex_discreted) telescope onto this line, so T_coex = T0/lambda and P_coex = P_S/lambda
    must lie on it to rounding at every step.  Using dV/dU for dU/dV, or the opposite sign,
    or the phases the other way round in only one of the two differences, leaves the line."""
    T0, P0 = 400.0, 13.0 / O.EV_A3_TO_GPA
    a = _FrozenPhase(8000, -4.25, 20.0)          # cd-like: higher energy, larger volume
    b = _FrozenPhase(7448, -4.21, 18.5)
    du, dv = -4.25 - (-4.21), 20.0 - 18.5
    if mode == O.DCCI_TEMP:
        pair = O.DcciPair(a, b, T0, P0, mode, T0, 1250.0, 1000)
    else:
        pair = O.DcciPair(a, b, T0, P0, mode, P0, 5.0 / O.EV_A3_TO_GPA, 1000)
    for _ in range(1000):
        pair.step()
        T, P = pair.coexistence()
        exact = T * (P0 / T0 - (du / dv) * (1.0 / T - 1.0 / T0))
        assert P == pytest.approx(exact, rel=1e-10, abs=1e-14)
        if mode == O.DCCI_TEMP:
            assert T == pytest.approx(pair.control(pair.k), rel=1e-12)
        else:
            assert P == pytest.approx(pair.control(pair.k), rel=1e-10)
    assert pair.error == 0


# ---------------------------------------------------------------- Uhlenbeck-Ford fluid reference
UF = (25.0, 2.0, 2200.0, 8.0)      # p, sigma (A), T_uf (K), rc (A): the liquid reference of Sec. 4


def _uf_dimer(r, rc=14.0):
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    return O.uf_energy(x, np.array([30.0, 30.0, 30.0]), (UF[0], UF[1], UF[2], rc))


def test_uf_second_virial_coefficient_closed_form():
    """B2 = -1/2 int (exp(-u/kT) - 1) d^3r: by quadrature of the oracle's own dimer energy
    (truncated at 7 sigma, where the Mayer function is e^-49) against the Gaussian-sum
    closed form, and the closed form against quadrature of (1 - exp(-r^2/sigma^2))^p - 1."""
    from scipy import integrate
    p, sig, T = UF[0], UF[1], UF[2]
    kT = O.KB * T
    b2 = O.uf_b2(int(p), sig)
    mayer = lambda r: (math.exp(-_uf_dimer(r)[0] / kT) - 1.0) * r * r
    q = integrate.quad(mayer, 1e-9, 14.0, limit=400, epsabs=1e-12, epsrel=1e-12)[0]
    assert -2.0 * math.pi * q == pytest.approx(b2, rel=1e-7)
    q2 = integrate.quad(lambda r: ((1.0 - math.exp(-(r / sig) ** 2)) ** p - 1.0) * r * r, 0.0, 30.0,
                        limit=400, epsabs=1e-13, epsrel=1e-13)[0]
    assert -2.0 * math.pi * q2 == pytest.approx(b2, rel=1e-10)
    # the potential is repulsive, continuous at rc and zero beyond
    e, f, _, _ = _uf_dimer(3.0, rc=8.0)
    assert e > 0.0 and f[1, 0] > 0.0 and f[0, 0] == -f[1, 0]
    assert _uf_dimer(8.0 - 1e-9, rc=8.0)[0] == pytest.approx(0.0, abs=1e-12)
    assert _uf_dimer(8.0 + 1e-9, rc=8.0)[0] == 0.0


def test_uf_third_virial_coefficient_closed_form():
    """B3 = -(8 pi^2 / 3) int int f(r) f(s) r^2 s^2 int_-1^1 f(sqrt(r^2 + s^2 - 2 r s c)) dc dr ds
    by Gauss-Legendre quadrature against the Gaussian-sum closed form."""
    p, sig = int(UF[0]), UF[1]
    f = lambda r: (1.0 - np.exp(-(r / sig) ** 2)) ** p - 1.0
    xr, wr = np.polynomial.legendre.leggauss(160)
    xc, wc = np.polynomial.legendre.leggauss(96)
    rmax = 6.0 * sig
    r = 0.5 * rmax * (xr + 1.0)
    w = 0.5 * rmax * wr
    R, S, C = np.meshgrid(r, r, xc, indexing="ij")
    inner = (f(np.sqrt(R * R + S * S - 2.0 * R * S * C)) * wc[None, None, :]).sum(axis=2)
    fr = f(r) * r * r * w
    b3 = -(8.0 * math.pi ** 2 / 3.0) * float(fr @ inner @ fr)
    assert b3 == pytest.approx(O.uf_b3(p, sig), rel=1e-6)


def test_uf_forces_and_virial_are_derivatives():
    x, box = I.liquid(300, 0.05, seed=12, rmin=1.0)
    e, f, vir, ea = O.uf_energy(x, box, UF)
    h = 1e-5
    fd = np.zeros_like(x)
    for i in range(0, len(x), 7):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd[i, k] = -(O.uf_energy(xp, box, UF)[0] - O.uf_energy(xm, box, UF)[0]) / (2 * h)
    sel = np.arange(0, len(x), 7)
    assert np.abs(fd[sel] - f[sel]).max() < 1e-6 * np.abs(f).max()
    assert np.abs(f.sum(axis=0)).max() < 1e-10
    assert ea.sum() == pytest.approx(e, rel=1e-12)
    # virial = -dE/d(strain): W_aa = -L_a dE/dL_a under affine scaling of axis a
    for a in range(3):
        s = np.ones(3); s[a] = 1.0 + h
        ep = O.uf_energy(x * s, box * s, UF)[0]
        s[a] = 1.0 - h
        em = O.uf_energy(x * s, box * s, UF)[0]
        assert vir[a] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-8)


def test_ideal_gas_free_energy_sackur_tetrode():
    """The classical ideal-gas free energy (the end state of the switching to the UF fluid)
    gives the Sackur-Tetrode entropy S = (U - F)/T: argon at 298.15 K and 1 bar against its
    tabulated standard entropy."""
    g = _golden("ideal_gas.txt")
    T, n = 298.15, 10 ** 6
    kT = O.KB * T
    e_charge, n_a = 1.602176634e-19, 6.02214076e23
    V = n * kT / (1e5 * 1e-30 / e_charge)          # 1 bar in eV/A^3
    F = O.ideal_gas_free_energy(n, V, T, g["argon_mass_g_per_mol"])
    S = (1.5 * n * kT - F) / T / n * e_charge * n_a
    assert S == pytest.approx(g["argon_S298_J_per_K_mol"], abs=0.005)


def _uf_switch_work(n, box, direction, seed, nsw):
    T = UF[2]
    x = np.random.default_rng(seed).uniform(0.0, 1.0, (n, 3)) * box
    pot = O.POT_EINSTEIN if direction > 0 else O.POT_UF
    eq = O.System(x=x, v=I.gaussian_velocities(n, _sv(T), seed), box=box.copy(), r0=x.copy(), pot=pot,
                  k_int=0.0, uf=UF, T=T, tdamp=0.1, seed=seed, sys_id=1)
    eq.run(500)
    sw = O.System(x=eq.x, v=eq.v, box=box.copy(), r0=x.copy(), pot=O.POT_EINSTEIN, k_int=0.0, ref=O.REF_UF,
                  uf=UF, T=T, tdamp=0.1, seed=seed, sys_id=2, sched=O.SCHED_FL, direction=direction, nsched=nsw)
    sw.run(nsw)
    return sw.W


def test_ideal_gas_to_uf_switching_follows_the_virial_series():
    """Hamiltonian interpolation from the ideal gas (lambda = 0) to the UF fluid (lambda = 1)
    at low density: the excess free energy of n atoms in a periodic box is
    F_ex / (n kT) = (n-1)/n rho B2 + (n-1)(n-2)/n^2 rho^2 B3 / 2 + O(rho^3) (pair and triplet
    counting of the cluster expansion).  At rho B2 = 0.2 the B3 term is 5 % of the total and
    the B4 term about 0.5 %; 8 + 8 realisations of 6000 steps, 128 atoms."""
    n, target = 128, 0.2
    p, sig, T = int(UF[0]), UF[1], UF[2]
    b2, b3 = O.uf_b2(p, sig), O.uf_b3(p, sig)
    rho = target / b2
    L = (n / rho) ** (1.0 / 3.0)
    box = np.array([L, L, L])
    reps, nsw = 8, 6000
    wf = np.array([_uf_switch_work(n, box, +1, s, nsw) for s in range(reps)])
    wb = np.array([_uf_switch_work(n, box, -1, 100 + s, nsw) for s in range(reps)])
    kT = O.KB * T
    fex = O.free_energy_difference(wf, wb) / (n * kT)
    sem = 0.5 * math.sqrt(wf.var(ddof=1) / reps + wb.var(ddof=1) / reps) / (n * kT)
    pred = (n - 1) / n * rho * b2 + (n - 1) * (n - 2) / n ** 2 * rho ** 2 * b3 / 2.0
    assert sem < 0.01
    assert abs(fex - pred) < 4.0 * sem + 0.002
    assert O.dissipated_heat(wf, wb) > 0.0
    # the free energy of the interacting fluid, Eq. dA with the ideal gas as reference
    f_uf = O.ideal_gas_free_energy(n, L ** 3, T) + O.free_energy_difference(wf, wb)
    assert f_uf > O.ideal_gas_free_energy(n, L ** 3, T)

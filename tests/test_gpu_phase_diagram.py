"""The paper's silicon phase-diagram chain (Sec. 4) run end to end through the C ABI.

Every dynamical step runs in the CUDA kernels (FP32 forces, FP64 integration and work); the
host only combines the work values with the estimators the paper states (the oracle's, which
are pinned on their own).  Shorter runs than the paper's (its 0.1-0.5 ns become 10-50 ps; the
work estimators and the dCCI line were checked to be converged at these lengths):

1. Si-cd at (400 K, 0 GPa) and Si-beta-tin at (400 K, 15 GPa): NPT for the mean box, then
   Frenkel-Ladd switching to the Einstein crystal (k = 6.113 / 1.362 eV/A^2), 10 forward and
   10 backward realisations: G = F_E - (W_f - W_b)/2 + P V (Sec. 2.1, Eq. dA, Eq. G_and_A).
2. Adiabatic switching in pressure, cd 0 -> 15 GPa and beta-tin 15 -> 5 GPa, forward and
   backward: G(P) along the path (Sec. 2.3, Eq. Gibbs_AS).  The crossing is the coexistence
   pressure at 400 K; at the paper's value the two Gibbs energies must agree within 2 meV/atom
   (1 meV/atom per phase, the free-energy tolerance).
3. dCCI in temperature control from (400 K, P_coex) to 1250 K over 100 ps, 10 coupled pairs
   (Sec. 3, Eq. Ps_coex_discreted): the coexistence line P(T).
4. Reversible scaling of both phases at P* = P_line(1210 K) from 400 K to 1250 K, forward and
   backward (Sec. 2.2, Eq. Gibbs_RS), starting from the step-2 Gibbs energies at P*: the two
   phases' G must cross where the dCCI line says, i.e. agree at 1210 K within 2 meV/atom.
   The two estimators share only the force kernels, so this checks the dCCI update, the
   barostat and the switching-work accumulation against each other.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_10449_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GPA = O.EV_A3_TO_GPA
T0 = 400.0
R = 10                                  # realisations per estimate (the paper's count)
NPT_STEPS, FL_STEPS, FL_EQ, AS_STEPS = 20000, 20000, 10000, 20000
DCCI_STEPS, DCCI_T1 = 100000, 1250.0
RS_STEPS = 50000
EVERY = 100
TOL_DG = 2e-3                           # eV/atom: 1 meV/atom for each of the two phases
LIQ_MELT, LIQ_NPT = 5000, 20000         # liquid: melting at 3000 K, NPT at 2200 K
UF_EQ, UF_STEPS = 5000, 40000           # ideal gas -> UF fluid (10k -> 40k steps moved F by 1.1 meV/atom)
HI_EQ, HI_STEPS = 5000, 30000           # SW liquid -> UF fluid (20k and 60k steps agree within 0.08 meV/atom)
LIQ_AS = 50000                          # liquid pressure switching 0 <-> 15 GPa
RS_EQ, RS_MELT = 10000, 100000          # reversible scaling through the melting points
DCCI_EQ, DCCI_MELT = 10000, 100000      # solid-liquid dCCI lines


def _golden():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "si_phase_diagram.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(v)
    return vals


PAPER = _golden()
SV = math.sqrt(O.KB * T0 / (O.M_SI * O.MVV2E))


@pytest.fixture(scope="module")
def N():
    from paper_2103_10449_gb300 import nefe
    nefe.load()
    return nefe


class Chain:
    """Runs the steps of the module docstring; every context holds all realisations."""

    def __init__(self, N):
        self.N = N
        xcd, bcd = I.diamond(10, 10, 10)
        xbs, bbs = I.beta_tin(*I.beta_tin_cells_for(8000))
        self.lat = {"cd": (xcd, bcd, N.NEFE_BARO_ISO), "bs": (xbs, bbs, N.NEFE_BARO_ANISO)}
        self.n = {"cd": len(xcd), "bs": len(xbs)}

    def ctx(self):
        return self.N.Context(precision=self.N.NEFE_FP32, dt=0.001, skin=0.7, nbr_cap=48)

    def npt(self, jobs, nsteps, nblocks, seed):
        """jobs: (phase, P_GPa, start, lambda0); start is a box scale for a fresh lattice or a
        list of R states.  Returns R states per job and the mean box over nblocks reads taken
        during nsteps further steps (None when nblocks = 0)."""
        N = self.N
        c = self.ctx()
        ids = []
        for j, (ph, P, start, lam0) in enumerate(jobs):
            x, b, mode = self.lat[ph]
            ss = []
            for r in range(R):
                if isinstance(start, list):
                    xs, vs, bs = start[r]
                else:
                    xs, bs, vs = x * start, b * start, I.gaussian_velocities(len(x), SV, seed + 1000 * j + r)
                s = c.add_system(xs, bs, v=vs)
                c.set_thermostat(s, T0, 0.1, seed + 1000 * j + r)
                c.set_barostat(s, mode, P, 1.0)
                if lam0 != 1.0:
                    c.set_schedule(s, N.NEFE_SCHED_NONE, lambda0=lam0)
                ss.append(s)
            ids.append(ss)
        c.run(nsteps)
        boxes = [[] for _ in jobs]
        for _ in range(nblocks):
            c.run(nsteps // nblocks)
            res = c.results_all()
            for j, ss in enumerate(ids):
                boxes[j] += [res[s]["box"] for s in ss]
        assert all(r["error"] == 0 for r in c.results_all())
        states = [[c.get_state(s) for s in ss] for ss in ids]
        c.close()
        return states, [np.mean(b, axis=0) if b else None for b in boxes]

    def _fl(self, sets, direction, extra):
        """Frenkel-Ladd switching of each (phase, r0, k_E, states) set; returns W per set and the
        final states (after `extra` further steps at the end point)."""
        N = self.N
        c = self.ctx()
        ids = []
        for j, (ph, r0, kE, states) in enumerate(sets):
            ss = []
            for r, (x, v, b) in enumerate(states):
                s = c.add_system(x, b, v=v, r0=r0)
                c.set_thermostat(s, T0, 0.1, (9000 if direction > 0 else 11000) + 100 * j + r)
                c.set_schedule(s, N.NEFE_SCHED_FL, direction=direction, nsteps=FL_STEPS, k_E=kE)
                ss.append(s)
            ids.append(ss)
        c.run(FL_STEPS)
        res = c.results_all()
        W = [np.array([res[s]["W"] for s in ss]) for ss in ids]
        if extra:
            c.run(extra)
        assert all(r["error"] == 0 for r in c.results_all())
        out = [[c.get_state(s) for s in ss] for ss in ids]
        c.close()
        return W, out

    def gibbs_400K(self):
        """Steps 1 and 2: G(P)/N of both phases at 400 K on a 5..15 GPa grid."""
        N = self.N
        st, mb = self.npt([("cd", 0.0, 1.0, 1.0), ("cd", 15.0, 0.96, 1.0), ("bs", 15.0, 1.0, 1.0),
                           ("bs", 5.0, 1.03, 1.0)], NPT_STEPS, 40, seed=1)
        c = self.ctx()
        fl = []
        for ph, j, kE in (("cd", 0, PAPER["k_einstein_cd"]), ("bs", 2, PAPER["k_einstein_betasn"])):
            x0, b0, _ = self.lat[ph]
            r0 = x0 * (mb[j] / b0)               # Einstein sites: the lattice at the mean box
            ss = []
            for r, (x, v, b) in enumerate(st[j]):
                xs = x * (mb[j] / b)
                xs += r0.mean(axis=0) - xs.mean(axis=0)
                s = c.add_system(xs, mb[j], v=v - v.mean(axis=0), r0=r0)
                c.set_thermostat(s, T0, 0.1, 5000 + 100 * j + r)
                ss.append(s)
            fl.append((ph, r0, kE, ss))
        sw = []                                  # AS runs share the NVT equilibration's context
        for j, P0, P1 in ((0, 0.0, 15.0), (1, 15.0, 0.0), (2, 15.0, 5.0), (3, 5.0, 15.0)):
            ss = []
            for r, (x, v, b) in enumerate(st[j]):
                s = c.add_system(x, b, v=v)
                c.set_thermostat(s, T0, 0.1, 7000 + 100 * j + r)
                c.set_barostat(s, self.lat["cd" if j < 2 else "bs"][2], P0, 1.0)
                c.set_schedule(s, N.NEFE_SCHED_AS, nsteps=AS_STEPS, P0_GPa=P0, P1_GPa=P1)
                c.set_trace(s, EVERY, AS_STEPS // EVERY + 16)
                ss.append(s)
            sw.append(ss)
        c.run(max(AS_STEPS, FL_EQ) + 2 * EVERY)
        assert all(r["error"] == 0 for r in c.results_all())
        tr = [[c.trace(s) for s in ss] for ss in sw]
        eq = [[c.get_state(s) for s in f[3]] for f in fl]
        c.close()
        Wf, at1 = self._fl([(ph, r0, kE, e) for (ph, r0, kE, _), e in zip(fl, eq)], 1, FL_EQ)
        Wb, _ = self._fl([(ph, r0, kE, e) for (ph, r0, kE, _), e in zip(fl, at1)], -1, 0)
        g0 = {}
        for k, (ph, j, P) in enumerate((("cd", 0, 0.0), ("bs", 2, 15.0))):
            n = self.n[ph]
            F = O.helmholtz_from_switching(O.einstein_free_energy(n, fl[k][2], T0), Wf[k].mean(), Wb[k].mean())
            g0[ph] = O.gibbs_from_helmholtz(F, P / GPA, float(np.prod(mb[j])))
        self.g0 = g0                             # G of cd at (400 K, 0 GPa), beta-tin at (400 K, 15 GPa)
        self.st400 = {"cd": st[0], "bs": st[2]}
        self.P = np.linspace(5.0, 15.0, 2001)
        self.G400 = {}
        for ph, f, b, P0 in (("cd", tr[0], tr[1], 0.0), ("bs", tr[2], tr[3], 15.0)):
            wf, wb = self._as_work(f, b, P0)
            self.G400[ph] = O.gibbs_as(g0[ph], wf, wb) / self.n[ph]
        return self.P, self.G400["cd"] - self.G400["bs"]

    def _as_work(self, fwd, bwd, P0):
        """Mean W(P0 -> P) of the forward runs and W(P -> P0) of the backward runs on self.P,
        read from the traces (column 7 is the target pressure, column 2 the work)."""
        a, b = [], []
        for tf, tb in zip(fwd, bwd):
            tf, tb = tf[tf[:, 0] <= AS_STEPS], tb[tb[:, 0] <= AS_STEPS]
            assert tf[0, 0] == 0 and tf[-1, 0] == AS_STEPS and tb[-1, 0] == AS_STEPS
            s = 1.0 if tf[-1, 7] > P0 else -1.0
            a.append(np.interp(s * self.P, s * tf[:, 7], tf[:, 2]))
            b.append(tb[-1, 2] - np.interp(-s * self.P, -s * tb[:, 7], tb[:, 2]))
        return np.mean(a, axis=0), np.mean(b, axis=0)

    def dcci_line(self, P_coex):
        """Step 3: mean coexistence pressure P(T) on 400..1250 K over R coupled pairs."""
        N = self.N
        st, _ = self.npt([("cd", P_coex, 0.965, 1.0), ("bs", P_coex, 1.0, 1.0)], NPT_STEPS, 0, seed=3)
        c = self.ctx()
        first = []
        for r in range(R):
            a = c.add_system(st[0][r][0], st[0][r][2], v=st[0][r][1])
            b = c.add_system(st[1][r][0], st[1][r][2], v=st[1][r][1])
            c.set_thermostat(a, T0, 0.1, 50 + 2 * r)
            c.set_thermostat(b, T0, 0.1, 51 + 2 * r)
            c.set_barostat(a, N.NEFE_BARO_ISO, P_coex, 1.0)
            c.set_barostat(b, N.NEFE_BARO_ANISO, P_coex, 1.0)
            c.pair_dcci(a, b, T0, P_coex, N.NEFE_DCCI_TEMP, T0, DCCI_T1, DCCI_STEPS)
            c.set_trace(a, 500, DCCI_STEPS // 500 + 8)
            first.append(a)
        c.run(DCCI_STEPS)
        assert all(r["error"] == 0 for r in c.results_all())
        self.T = np.linspace(T0, DCCI_T1, 851)
        lines = []
        for a in first:
            t = c.trace(a)
            t = t[t[:, 0] <= DCCI_STEPS]
            # physical state of the scaled pair: T = T0 / lambda, P = P_S / lambda
            lines.append(np.interp(self.T, T0 / t[:, 1], t[:, 7] / t[:, 1]))
        self.dcci_states = st
        c.close()
        self.ss_line = (self.T, np.mean(lines, axis=0))
        return self.ss_line

    def rs_gibbs(self, P_star):
        """Step 4: G(T)/N of both phases at P_star on 400..1250 K by reversible scaling, from
        the 400 K Gibbs energies of step 2 (backward runs start equilibrated at lambda_f)."""
        N = self.N
        lam_f = T0 / DCCI_T1
        st = self.dcci_states
        eq, _ = self.npt([("cd", P_star, st[0], 1.0), ("bs", P_star, st[1], 1.0),
                          ("cd", lam_f * P_star, st[0], lam_f), ("bs", lam_f * P_star, st[1], lam_f)],
                         NPT_STEPS, 0, seed=5)
        c = self.ctx()
        ids = []
        for j, (ph, direction) in enumerate((("cd", 1), ("bs", 1), ("cd", -1), ("bs", -1))):
            ss = []
            for r, (x, v, b) in enumerate(eq[j]):
                s = c.add_system(x, b, v=v)
                c.set_thermostat(s, T0, 0.1, 13000 + 100 * j + r)
                c.set_barostat(s, self.lat[ph][2], P_star if direction > 0 else lam_f * P_star, 1.0)
                c.set_schedule(s, N.NEFE_SCHED_RS, direction=direction, nsteps=RS_STEPS, lambda_f=lam_f,
                               P_GPa=P_star)
                c.set_trace(s, EVERY, RS_STEPS // EVERY + 16)
                ss.append(s)
            ids.append(ss)
        c.run(RS_STEPS + 2 * EVERY)
        assert all(r["error"] == 0 for r in c.results_all())
        tr = [[c.trace(s) for s in ss] for ss in ids]
        c.close()
        lam = np.linspace(1.0, lam_f, 2001)
        G = {}
        for k, ph in enumerate(("cd", "bs")):
            n = self.n[ph]
            g0 = float(np.interp(P_star, self.P, self.G400[ph])) * n
            a, b = [], []
            for tf, tb in zip(tr[k], tr[k + 2]):
                tf, tb = tf[tf[:, 0] <= RS_STEPS], tb[tb[:, 0] <= RS_STEPS]
                assert tf[-1, 0] == RS_STEPS and tf[-1, 1] == pytest.approx(lam_f, abs=1e-12)
                a.append(np.interp(-lam, -tf[:, 1], tf[:, 2]))               # W(1 -> lambda)
                b.append(tb[-1, 2] - np.interp(lam, tb[:, 1], tb[:, 2]))      # W(lambda -> 1)
            G[ph] = O.gibbs_rs(g0, n, T0, lam, np.mean(a, axis=0), np.mean(b, axis=0)) / n
        return T0 / lam, G["cd"] - G["bs"]


class LiquidChain:
    """The liquid half of the phase diagram (Sec. 4): the liquid's absolute Gibbs energy from the
    Uhlenbeck-Ford reference, its G(T) at 0 and 15 GPa by reversible scaling, the solids' G(T)
    by reversible scaling from their 400 K Gibbs energies, the melting points at the crossings,
    and the two solid-liquid dCCI lines.  Liquid steps (L*) run at T_L = 2200 K:

    L1. NPT of the liquid (8000 atoms, melted from random positions at 3000 K) for the mean box.
    L2. The UF fluid's free energy at that box: switching from the ideal gas (lambda 0 -> 1 of
        H = (1 - lambda) * 0 + lambda U_UF), F_UF = F_ideal + (W_f - W_b)/2.
    L3. Hamiltonian interpolation SW liquid -> UF fluid: F_liq = F_UF - (W_f - W_b)/2 (Eq. dA);
        G = F + P V (Eq. G_and_A).
    L4. Adiabatic switching in pressure 0 -> 15 GPa at T_L (Eq. Gibbs_AS): G_liq(15 GPa, T_L).
    L5. Reversible scaling at 0 GPa (T_L -> 1200 K) and at 15 GPa (T_L -> 1100 K) with the
        barostat target lambda P (Eq. Gibbs_RS); the solids from 400 K to 2000 K (Si-cd, 0 GPa) and
        1600 K (beta-tin, 15 GPa).  The paper cools the liquid to 800 K and 1000 K; stopping
        above 1100 K keeps the supercooled liquid fast-relaxing over the part of the path that
        reaches the melting points (1689 K and 1365 K).
    """

    UF = (25.0, 2.0, 2200.0, 8.0)
    T_L = 2200.0

    def __init__(self, N, solid):
        self.N, self.solid = N, solid
        self.n = 8000
        self.sv = math.sqrt(O.KB * self.T_L / (O.M_SI * O.MVV2E))

    def ctx(self):
        return self.N.Context(precision=self.N.NEFE_FP32, dt=0.001, skin=0.7, nbr_cap=48)

    def liquid_states(self, P, seed, nsteps=LIQ_NPT):
        """R liquid states at (T_L, P) after melting at 3000 K and NPT at T_L; their mean box."""
        N = self.N
        c = self.ctx()
        x0, b0 = I.liquid(self.n, 0.05425, seed=seed)
        ss = []
        for r in range(R):
            s = c.add_system(x0, b0, v=I.gaussian_velocities(self.n, self.sv, seed + r))
            c.set_thermostat(s, 3000.0, 0.1, seed + 100 + r)
            ss.append(s)
        c.run(LIQ_MELT)
        st = [c.get_state(s) for s in ss]
        c.close()
        c = self.ctx()
        ss = []
        for r, (x, v, b) in enumerate(st):
            s = c.add_system(x, b, v=v * math.sqrt(self.T_L / 3000.0))
            c.set_thermostat(s, self.T_L, 0.1, seed + 200 + r)
            c.set_barostat(s, N.NEFE_BARO_ISO, P, 1.0)
            ss.append(s)
        c.run(nsteps)
        boxes = []
        for _ in range(20):
            c.run(nsteps // 20)
            boxes += [c.results(s)["box"] for s in ss]
        assert all(r["error"] == 0 for r in c.results_all())
        st = [c.get_state(s) for s in ss]
        c.close()
        return st, np.mean(boxes, axis=0)

    def f_uf(self, box, nsw=UF_STEPS):
        """L2: Helmholtz free energy of the UF fluid of n atoms in `box` at T_L."""
        N = self.N
        uf = N.uf_params(*self.UF)
        L = box
        eq = self.ctx()
        for r in range(R):
            x = np.random.default_rng(2000 + r).uniform(0.0, 1.0, (self.n, 3)) * L
            s = eq.add_system(x, L, v=I.gaussian_velocities(self.n, self.sv, 2100 + r), pot=N.NEFE_POT_UF)
            eq.set_uf_params(s, uf)
            eq.set_thermostat(s, self.T_L, 0.1, 2200 + r)
        eq.run(UF_EQ)
        ufst = [eq.get_state(s)[:2] for s in range(R)]
        eq.close()
        c = self.ctx()
        for r in range(2 * R):
            if r < R:
                x = np.random.default_rng(2300 + r).uniform(0.0, 1.0, (self.n, 3)) * L
                v = I.gaussian_velocities(self.n, self.sv, 2400 + r)
            else:
                x, v = ufst[r - R]
            s = c.add_system(x, L, v=v, r0=x, pot=N.NEFE_POT_EINSTEIN, k_int=0.0)
            c.set_uf_params(s, uf)
            c.set_thermostat(s, self.T_L, 0.1, 2500 + r)
            c.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if r < R else -1, nsteps=nsw, ref=N.NEFE_REF_UF)
        c.run(nsw)
        res = c.results_all()
        c.close()
        assert all(r["error"] == 0 for r in res)
        wf = np.array([res[r]["W"] for r in range(R)])
        wb = np.array([res[r]["W"] for r in range(R, 2 * R)])
        f_id = O.ideal_gas_free_energy(self.n, float(np.prod(L)), self.T_L)
        return f_id + O.free_energy_difference(wf, wb), wf, wb

    def f_liquid(self, states, box, f_uf, nsw=HI_STEPS):
        """L3: Helmholtz free energy of the SW liquid at `box` and T_L (Eq. dA, UF reference)."""
        N = self.N
        uf = N.uf_params(*self.UF)
        c = self.ctx()
        ids = []
        for r, (x, v, b) in enumerate(states):
            xs = x * (box / b)
            s = c.add_system(xs, box, v=v)
            c.set_uf_params(s, uf)
            c.set_thermostat(s, self.T_L, 0.1, 2600 + r)
            ids.append(s)
        c.run(HI_EQ)
        st = [c.get_state(s) for s in ids]
        c.close()
        eq = self.ctx()                          # UF end states for the backward runs
        for r, (x, v, b) in enumerate(st):
            s = eq.add_system(x, box, v=v, pot=N.NEFE_POT_UF)
            eq.set_uf_params(s, uf)
            eq.set_thermostat(s, self.T_L, 0.1, 2700 + r)
        eq.run(HI_EQ)
        ufst = [eq.get_state(s) for s in range(R)]
        eq.close()
        c = self.ctx()
        for r in range(2 * R):
            x, v, _ = st[r] if r < R else ufst[r - R]
            s = c.add_system(x, box, v=v)
            c.set_uf_params(s, uf)
            c.set_thermostat(s, self.T_L, 0.1, 2800 + r)
            c.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if r < R else -1, nsteps=nsw, ref=N.NEFE_REF_UF)
        c.run(nsw)
        res = c.results_all()
        c.close()
        assert all(r["error"] == 0 for r in res)
        wf = np.array([res[r]["W"] for r in range(R)])
        wb = np.array([res[r]["W"] for r in range(R, 2 * R)])
        return O.helmholtz_from_switching(f_uf, wf, wb), wf, wb

    def equilibrate(self, jobs, nsteps, seed):
        """jobs: (states, barostat mode, P_GPa, T, lambda0); NPT at (T, lambda0 P) with the
        potential scaled by lambda0 (the end state of a reversible-scaling path)."""
        N = self.N
        c = self.ctx()
        ids = []
        for j, (states, mode, P, T, lam0) in enumerate(jobs):
            ss = []
            for r, (x, v, b) in enumerate(states):
                s = c.add_system(x, b, v=v)
                c.set_thermostat(s, T, 0.1, seed + 1000 * j + r)
                c.set_barostat(s, mode, lam0 * P, 1.0)
                if lam0 != 1.0:
                    c.set_schedule(s, N.NEFE_SCHED_NONE, lambda0=lam0)
                ss.append(s)
            ids.append(ss)
        c.run(nsteps)
        assert all(r["error"] == 0 for r in c.results_all())
        out = [[c.get_state(s) for s in ss] for ss in ids]
        c.close()
        return out

    def rs(self, jobs, nsteps, seed):
        """Reversible scaling (Eq. Gibbs_RS) of each job (fwd states at lambda 1, bwd states at
        lambda_f, barostat mode, P_GPa, T0, lambda_f, G0 (eV, whole system), n): G(T)/N on a
        grid of T = T0/lambda from lambda 1 to lambda_f."""
        N = self.N
        c = self.ctx()
        ids = []
        for j, (fw, bw, mode, P, T0_, lam_f, _, _) in enumerate(jobs):
            pair = []
            for direction, states in ((1, fw), (-1, bw)):
                ss = []
                for r, (x, v, b) in enumerate(states):
                    s = c.add_system(x, b, v=v)
                    c.set_thermostat(s, T0_, 0.1, seed + 1000 * j + 100 * (direction > 0) + r)
                    c.set_barostat(s, mode, P if direction > 0 else lam_f * P, 1.0)
                    c.set_schedule(s, N.NEFE_SCHED_RS, direction=direction, nsteps=nsteps, lambda_f=lam_f, P_GPa=P)
                    c.set_trace(s, EVERY, nsteps // EVERY + 16)
                    ss.append(s)
                pair.append(ss)
            ids.append(pair)
        c.run(nsteps + 2 * EVERY)
        assert all(r["error"] == 0 for r in c.results_all())
        out = []
        for (fw, bw, mode, P, T0_, lam_f, g0, n), (sf, sb) in zip(jobs, ids):
            lam = np.linspace(1.0, lam_f, 2001)
            sgn = 1.0 if lam_f > 1.0 else -1.0
            a, b = [], []
            for s1, s2 in zip(sf, sb):
                tf, tb = c.trace(s1), c.trace(s2)
                tf, tb = tf[tf[:, 0] <= nsteps], tb[tb[:, 0] <= nsteps]
                assert tf[-1, 0] == nsteps and tf[-1, 1] == pytest.approx(lam_f, abs=1e-12)
                a.append(np.interp(sgn * lam, sgn * tf[:, 1], tf[:, 2]))                 # W(1 -> lambda)
                b.append(tb[-1, 2] - np.interp(-sgn * lam, -sgn * tb[:, 1], tb[:, 2]))   # W(lambda -> 1)
            G = O.gibbs_rs(g0, n, T0_, lam, np.mean(a, axis=0), np.mean(b, axis=0)) / n
            out.append((T0_ / lam, G))
        c.close()
        return out

    def gibbs_liquid(self):
        """L1-L4: G/N of the liquid at (T_L, 0 GPa) and (T_L, 15 GPa), and the states there."""
        N = self.N
        n = self.n
        st0, box0 = self.liquid_states(0.0, seed=31)
        f_uf0, uwf, uwb = self.f_uf(box0)
        self.uf_w = (uwf, uwb)
        self.f_uf0 = f_uf0
        f_liq, wf, wb = self.f_liquid(st0, box0, f_uf0)
        self.hi_w = (wf, wb)
        self.g_liq0 = O.gibbs_from_helmholtz(f_liq, 0.0, float(np.prod(box0))) / n
        st15, _ = self.liquid_states(15.0, seed=37)
        # L4: pressure switching 0 -> 15 GPa and back at T_L (Eq. Gibbs_AS)
        c = self.ctx()
        fw, bw = [], []
        for r in range(R):
            for states, P0, P1, lst in ((st0, 0.0, 15.0, fw), (st15, 15.0, 0.0, bw)):
                x, v, b = states[r]
                s = c.add_system(x, b, v=v)
                c.set_thermostat(s, self.T_L, 0.1, 3000 + 10 * r + len(lst))
                c.set_barostat(s, N.NEFE_BARO_ISO, P0, 1.0)
                c.set_schedule(s, N.NEFE_SCHED_AS, nsteps=LIQ_AS, P0_GPa=P0, P1_GPa=P1)
                lst.append(s)
        c.run(LIQ_AS)
        res = c.results_all()
        c.close()
        assert all(r["error"] == 0 for r in res)
        w_up = np.mean([res[s]["W"] for s in fw])
        w_down = np.mean([res[s]["W"] for s in bw])
        self.g_liq15 = float(O.gibbs_as(self.g_liq0 * n, w_up, w_down)) / n
        self.liq_states = {0.0: st0, 15.0: st15}
        return self.g_liq0, self.g_liq15

    def melting(self, P):
        """Melting point at P (0 GPa: Si-cd; 15 GPa: Si-beta-tin) from the crossing of the solid's
        and the liquid's G(T) by reversible scaling (the solid from 400 K, the liquid from T_L)."""
        N = self.N
        ch = self.solid
        ph, mode, t_hi = ("cd", N.NEFE_BARO_ISO, 2000.0) if P == 0.0 else ("bs", N.NEFE_BARO_ANISO, 1600.0)
        t_lo = 1200.0 if P == 0.0 else 1100.0
        lam_s, lam_l = T0 / t_hi, self.T_L / t_lo
        sol = ch.st400[ph]
        liq = self.liq_states[P]
        eq = self.equilibrate([(sol, mode, P, T0, lam_s), (liq, N.NEFE_BARO_ISO, P, self.T_L, lam_l)],
                              RS_EQ, seed=4000 + int(P))
        g_liq = self.g_liq0 if P == 0.0 else self.g_liq15
        (Ts, Gs), (Tl, Gl) = self.rs([(sol, eq[0], mode, P, T0, lam_s, ch.g0[ph], ch.n[ph]),
                                      (liq, eq[1], N.NEFE_BARO_ISO, P, self.T_L, lam_l, g_liq * self.n, self.n)],
                                     RS_MELT, seed=5000 + int(P))
        T = np.linspace(t_lo, t_hi, 801)
        dG = np.interp(T, Ts, Gs) - np.interp(T, Tl[::-1], Gl[::-1])
        return T, dG

    def dcci_melting_line(self, T_m, P0, P1, solid_mode, seed):
        """dCCI in pressure control (Eq. l_coex_discreted) of R solid/liquid pairs from the
        coexistence point (T_m, P0) to P1: mean T_coex(P) on a grid of P."""
        N = self.N
        ch = self.solid
        ph = "cd" if P0 == 0.0 else "bs"
        eq = self.equilibrate([(ch.st400[ph], solid_mode, P0, T_m, 1.0),
                               (self.liq_states[P0], N.NEFE_BARO_ISO, P0, T_m, 1.0)], DCCI_EQ, seed=seed)
        c = self.ctx()
        first = []
        for r in range(R):
            a = c.add_system(eq[0][r][0], eq[0][r][2], v=eq[0][r][1])
            b = c.add_system(eq[1][r][0], eq[1][r][2], v=eq[1][r][1])
            c.set_thermostat(a, T_m, 0.1, seed + 2 * r)
            c.set_thermostat(b, T_m, 0.1, seed + 2 * r + 1)
            c.set_barostat(a, solid_mode, P0, 1.0)
            c.set_barostat(b, N.NEFE_BARO_ISO, P0, 1.0)
            c.pair_dcci(a, b, T_m, P0, N.NEFE_DCCI_PRESS, P0, P1, DCCI_MELT)
            c.set_trace(a, 500, DCCI_MELT // 500 + 8)
            first.append(a)
        c.run(DCCI_MELT)
        assert all(r["error"] == 0 for r in c.results_all())
        P = np.linspace(min(P0, P1), max(P0, P1), 501)
        lines = []
        for a in first:
            t = c.trace(a)
            t = t[t[:, 0] <= DCCI_MELT]
            Pt, Tt = t[:, 7] / t[:, 1], T_m / t[:, 1]          # P = P_S / lambda, T = T0 / lambda
            o = np.argsort(Pt)
            lines.append(np.interp(P, Pt[o], Tt[o]))
        c.close()
        return P, np.mean(lines, axis=0)


def _root(x, y):
    k = np.where(np.sign(y[:-1]) != np.sign(y[1:]))[0]
    assert len(k), "no crossing"
    k = int(k[0])
    return float(x[k] - y[k] * (x[k + 1] - x[k]) / (y[k + 1] - y[k]))


@pytest.fixture(scope="module")
def chain(N):
    ch = Chain(N)
    P, dG = ch.gibbs_400K()
    ch.P_coex = _root(P, dG)
    ch.dG_paper = float(np.interp(PAPER["p_coex_cd_betasn_400K"], P, dG))
    return ch


def test_coexistence_pressure_at_400K_matches_paper(chain):
    """Gibbs energies of Si-cd and Si-beta-tin at the paper's 400 K coexistence pressure agree
    within 2 meV/atom (0.22 GPa at the volume difference of about 1.45 A^3/atom)."""
    print(f"P_coex(400 K) = {chain.P_coex:.4f} GPa; G_cd - G_beta-tin at "
          f"{PAPER['p_coex_cd_betasn_400K']} GPa = {1e3 * chain.dG_paper:.3f} meV/atom")
    assert abs(chain.dG_paper) <= TOL_DG
    # cd is the stable phase below the crossing, beta-tin above it
    i5, i15 = 0, len(chain.P) - 1
    assert chain.G400["cd"][i5] < chain.G400["bs"][i5] and chain.G400["cd"][i15] > chain.G400["bs"][i15]


def test_dcci_line_agrees_with_reversible_scaling(chain):
    """The dCCI line through (400 K, P_coex) and the reversible-scaling Gibbs energies at the
    line's 1210 K pressure agree: G_cd - G_beta-tin there within 2 meV/atom."""
    T, line = chain.dcci_line(chain.P_coex)
    Tx = PAPER["triple_point_T"]
    P_star = float(np.interp(Tx, T, line))
    assert np.all(np.diff(line[::50]) < 0.0)    # the solid-solid line falls with temperature
    Ts, dG = chain.rs_gibbs(P_star)
    dG_x = float(np.interp(Tx, Ts, dG))
    print(f"dCCI P({Tx:.0f} K) = {P_star:.3f} GPa (paper's triple point {PAPER['triple_point_P']} GPa); "
          f"RS G_cd - G_beta-tin there = {1e3 * dG_x:.3f} meV/atom; RS crossing at {_root(Ts, dG):.1f} K")
    assert abs(dG_x) <= TOL_DG


@pytest.fixture(scope="module")
def liquid(N, chain):
    lc = LiquidChain(N, chain)
    lc.gibbs_liquid()
    lc.tm = {}
    return lc


def _melting(liquid, P):
    if P not in liquid.tm:
        T, dG = liquid.melting(P)
        liquid.tm[P] = (_root(T, dG), T, dG)
    return liquid.tm[P]


@pytest.mark.parametrize("P,key", [(0.0, "t_m_cd_0GPa"), (15.0, "t_m_betasn_15GPa")])
def test_melting_point_matches_paper(liquid, P, key):
    """The liquid's Gibbs energy from the UF reference (L1-L3, with the UF fluid's own free energy
    from the ideal gas) and reversible scaling crosses the solid's at the paper's melting point:
    G_solid - G_liquid there within 2 meV/atom (1 meV/atom per phase; about 11 K at the entropy of
    melting of SW silicon)."""
    Tm, T, dG = _melting(liquid, P)
    dG_paper = float(np.interp(PAPER[key], T, dG))
    print(f"P = {P} GPa: T_m = {Tm:.1f} K (paper {PAPER[key]} K); G_solid - G_liquid at the paper's T_m = "
          f"{1e3 * dG_paper:.3f} meV/atom; G_liq(2200 K, 0 GPa) = {liquid.g_liq0:.5f} eV/atom, "
          f"G_liq(2200 K, 15 GPa) = {liquid.g_liq15:.5f} eV/atom")
    assert abs(dG_paper) <= TOL_DG
    assert dG[0] < 0.0 < dG[-1]          # the solid is stable below T_m, the liquid above


def test_solid_liquid_dcci_lines_and_triple_point(liquid, chain, N):
    """dCCI in pressure control along the two melting lines (Si-cd/liquid 0 -> 10.2 GPa from
    (T_m, 0 GPa); Si-beta-tin/liquid 15 -> 9.4 GPa from (T_m, 15 GPa); 100 ps each, 10 pairs) and
    the solid-solid line of the first chain: the melting lines cross at the triple point, which
    the solid-solid line must pass through (within 2 meV/atom, i.e. about 15 K / 0.3 GPa); the
    paper's triple point is 1210(2) K, 9.90(3) GPa."""
    tm0 = _melting(liquid, 0.0)[0]
    tm15 = _melting(liquid, 15.0)[0]
    Pa, Ta = liquid.dcci_melting_line(tm0, 0.0, 10.2, N.NEFE_BARO_ISO, seed=6000)
    Pb, Tb = liquid.dcci_melting_line(tm15, 15.0, 9.4, N.NEFE_BARO_ANISO, seed=6100)
    P = np.linspace(9.4, 10.2, 401)
    d = np.interp(P, Pa, Ta) - np.interp(P, Pb, Tb)
    Pt = _root(P, d)
    Tt = float(np.interp(Pt, Pa, Ta))
    if not hasattr(chain, "ss_line"):
        chain.dcci_line(chain.P_coex)
    Ts, Ps = chain.ss_line
    P_ss = float(np.interp(Tt, Ts, Ps))
    print(f"melting lines: cd/liquid T(0) = {Ta[0]:.1f} K, T(10.2 GPa) = {Ta[-1]:.1f} K; beta-tin/liquid "
          f"T(9.4 GPa) = {Tb[0]:.1f} K, T(15 GPa) = {Tb[-1]:.1f} K; triple point {Tt:.1f} K, {Pt:.3f} GPa "
          f"(paper {PAPER['triple_point_T']} K, {PAPER['triple_point_P']} GPa); solid-solid line at {Tt:.0f} K: "
          f"{P_ss:.3f} GPa")
    assert np.all(np.diff(Ta[::25]) < 0.0)      # Si-cd melts at lower T under pressure (denser liquid)
    assert abs(P_ss - Pt) <= 0.3
    assert abs(Tt - PAPER["triple_point_T"]) <= 15.0 and abs(Pt - PAPER["triple_point_P"]) <= 0.3

"""FP64 CPU oracle for the non-equilibrium free-energy / dCCI hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It shares no code with the CUDA library in ``paper_2103_10449_gb300``
and never imports it; inputs come from ``paper_2103_10449_gb300.inputs`` (seeded generators
with none of the method's arithmetic) or from the caller.

The O(N^2) Stillinger-Weber energy/force/virial, the brute-force neighbour list, the cell
sort and the Philox noise live in ``nefe_oracle.c`` (compiled with ``-ffp-contract=off``);
this module wraps them with ctypes and writes out, step by step, what the paper computes:

* Hamiltonian interpolation and its driving force (Sec. 2.1, Eqs. H_lambda, Wrev_HI, dA);
* reversible scaling in NPT (Sec. 2.2, Eqs. H_RS, T_sc, P_sc, dH_RS, Gibbs_RS) and the Gibbs
  / Helmholtz relation (Eq. G_and_A);
* adiabatic switching in pressure (Sec. 2.3, Eqs. Wmech_dyn, Gibbs_AS);
* the dynamical work, left-point discretised (Eq. Wdyn; the same discretisation the paper
  uses for dCCI in Eq. Ps_coex_discreted);
* the forward/backward estimators (Eqs. dF, Qdiss);
* the discrete dCCI updates in temperature control (Eq. Ps_coex_discreted) and pressure
  control (Eq. l_coex_discreted) (Sec. 3);
* velocity-Verlet with a Langevin thermostat whose net random force is removed, and a
  Parrinello-Rahman-type box equation whose target pressure is multiplied by lambda
  (Sec. 4: "Langevin thermostat", "velocity-Verlet", dt = 1 fs, the ``ners`` tag).

Where the paper is silent, the reading taken is stated in the docstring of the routine
that implements it.

Parity status: the SW energy/forces, neighbour list, cells, Philox, Einstein free energy,
integrator, thermostat, schedules, estimators (including the sign of Eq. dA) and the dCCI
updates (against the exact Clausius-Clapeyron line for constant dU, dV) are pinned by tests
in ``tests/test_oracle_pins.py``.  The barostat equation is a reading (the paper names
Parrinello-Rahman but gives no equations).  Its equilibrium is pinned by closed forms:
pressure switching of an ideal gas reproduces (N - 1) kB T ln(P1/P0) for the isotropic and
the anisotropic form, and the anisotropic form relaxes each axis of a beta-Sn cell to the
static enthalpy minimum.  Its dynamics are pinned to the reading (the small-oscillation
frequency of the volume of an ideal gas); that reading itself has no counterpart in the
paper.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nefe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# --- physical constants (CODATA 2018) and metal units (A, eV, ps, g/mol, K) -------------
KB = 8.617333262e-5                       # eV / K
HBAR = 6.582119569e-4                     # eV ps
MVV2E = 1.66053906660e-27 * 1e4 / 1.602176634e-19   # (g/mol) A^2/ps^2 -> eV
EV_A3_TO_GPA = 1.602176634e-19 / 1e-30 / 1e9           # eV/A^3 -> GPa
M_SI = 28.0855                            # g/mol

# Standard Stillinger-Weber silicon parameters (Stillinger & Weber 1985), in the order
# eps, sigma, A, B, p, q, a, lambda3, gamma, cos(theta0).
SW_SI = (2.1683, 2.0951, 7.049556277, 0.6022245584, 4.0, 0.0, 1.80, 21.0, 1.20, -1.0 / 3.0)


def build(force: bool = False) -> str:
    """Compile nefe_oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                               _SRC, "-o", _LIB, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint64)
        lp = ctypes.POINTER(ctypes.c_int64)
        L.orc_philox4x64.argtypes = [up, up, up]
        L.orc_langevin_xi.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int64, dp]
        L.orc_sw_energy.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, dp]
        L.orc_sw_energy.restype = ctypes.c_double
        L.orc_sw_force_atoms.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int64, lp, dp]
        L.orc_neighbor_list.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_int,
                                        ip, ip, ip]
        L.orc_cell_bin.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_int,
                                   ip, ip, ip, ip]
        L.orc_uf_energy.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, dp]
        L.orc_uf_energy.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct))


# ------------------------------------------------------------------------------------------
# Wrapped C routines
# ------------------------------------------------------------------------------------------
def philox4x64(ctr, key):
    """Philox4x64-10 block for counter ``ctr`` (4 uint64) and key ``key`` (2 uint64)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_p(c, ctypes.c_uint64), _p(k, ctypes.c_uint64), _p(out, ctypes.c_uint64))
    return out


def langevin_xi(seed: int, sys_id: int, step: int, n: int) -> np.ndarray:
    """Standard-normal thermostat noise, shape (n, 3), counter (step, atom, sys, 0), key (seed, 0)."""
    xi = np.zeros((n, 3))
    lib().orc_langevin_xi(seed, sys_id, step, n, _p(xi))
    return xi


def sw_energy(x, box, prm=SW_SI):
    """Brute-force SW energy, forces (n,3), virial (xx,yy,zz,xy,xz,yz) and per-atom energy."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64)
    p = np.ascontiguousarray(prm, dtype=np.float64)
    f = np.zeros((n, 3))
    vir = np.zeros(6)
    ea = np.zeros(n)
    e = lib().orc_sw_energy(n, _p(x), _p(box), _p(p), _p(f), _p(vir), _p(ea))
    if math.isnan(e):
        raise ValueError("orc_sw_energy: box smaller than 2*a*sigma or neighbour shell overflow")
    return e, f, vir, ea


def sw_force_atoms(x, box, idx, prm=SW_SI):
    """Forces on the atoms ``idx`` only (each by its own brute-force neighbour search)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    box = np.ascontiguousarray(box, dtype=np.float64)
    p = np.ascontiguousarray(prm, dtype=np.float64)
    out = np.zeros((idx.size, 3))
    rc = lib().orc_sw_force_atoms(x.shape[0], _p(x), _p(box), _p(p), idx.size,
                                  _p(idx, ctypes.c_int64), _p(out))
    if rc != 0:
        raise ValueError("orc_sw_force_atoms failed")
    return out


def neighbor_list(x, box, rcs, cap=64):
    """Brute-force Verlet list: (nbr[n,cap], cnt[n], img[n,cap,3]); raises on overflow."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64)
    nbr = np.full((n, cap), -1, dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int32)
    img = np.zeros((n, cap, 3), dtype=np.int32)
    rc = lib().orc_neighbor_list(n, _p(x), _p(box), rcs, cap, _p(nbr, ctypes.c_int32),
                                 _p(cnt, ctypes.c_int32), _p(img, ctypes.c_int32))
    if rc == -2:
        raise ValueError("box length below 2*(rc+skin)")
    if rc == -1:
        raise OverflowError("neighbour row exceeds cap")
    return nbr, cnt, img


def cell_bin(x, box, rcs, ncell_cap=1 << 22):
    """Cell grid (3,), cell id per atom, cell_start (ncells+1,), perm (n,)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64)
    nc3 = np.zeros(3, dtype=np.int32)
    cell_of = np.zeros(n, dtype=np.int32)
    start = np.zeros(ncell_cap + 1, dtype=np.int32)
    perm = np.zeros(n, dtype=np.int32)
    tot = lib().orc_cell_bin(n, _p(x), _p(box), rcs, ncell_cap, _p(nc3, ctypes.c_int32),
                             _p(cell_of, ctypes.c_int32), _p(start, ctypes.c_int32),
                             _p(perm, ctypes.c_int32))
    if tot < 0:
        raise ValueError("cell grid below 2 cells per axis or above capacity")
    return nc3, cell_of, start[: tot + 1].copy(), perm


def uf_energy(x, box, uf):
    """Brute-force Uhlenbeck-Ford energy, forces (n,3), virial (xx,yy,zz,xy,xz,yz) and per-atom
    energy.  ``uf`` = (p, sigma, T_uf, rc): u(r) = -p kB T_uf ln(1 - exp(-r^2/sigma^2)) - u(rc) for
    r < rc (Sec. 2.1 names the UF model as the fluid reference; Sec. 4 uses p = 25, sigma = 2.0)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64)
    p = np.array([uf[0], uf[1], KB * uf[2], uf[3]], dtype=np.float64)
    f = np.zeros((n, 3))
    vir = np.zeros(6)
    ea = np.zeros(n)
    e = lib().orc_uf_energy(n, _p(x), _p(box), _p(p), _p(f), _p(vir), _p(ea))
    if math.isnan(e):
        raise ValueError("orc_uf_energy: box smaller than 2 rc")
    return e, f, vir, ea


# ------------------------------------------------------------------------------------------
# Closed forms and estimators
# ------------------------------------------------------------------------------------------
def _uf_mayer_coefficients(p: int):
    """The UF Mayer function exp(-u/kT) - 1 = (1 - exp(-r^2/sigma^2))^p - 1 expanded by the
    binomial theorem: sum_{k=1..p} C(p, k) (-1)^k exp(-k r^2/sigma^2) (integer p)."""
    if int(p) != p or p < 1:
        raise ValueError("the closed forms need an integer p >= 1")
    p = int(p)
    return [(k, math.comb(p, k) * (-1) ** k) for k in range(1, p + 1)]


def uf_b2(p: int, sigma: float) -> float:
    """Second virial coefficient of the untruncated UF fluid, B2 = -1/2 int f d^3r with the
    Gaussian expansion of the Mayer function: int exp(-k r^2/sigma^2) d^3r = (pi/k)^(3/2) sigma^3,
    so B2 = -(pi^(3/2) sigma^3 / 2) sum_k C(p,k) (-1)^k k^(-3/2)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    s = sum(Decimal(c) / (Decimal(k) * Decimal(k).sqrt()) for k, c in _uf_mayer_coefficients(p))
    return -0.5 * math.pi ** 1.5 * sigma ** 3 * float(s)


def uf_b3(p: int, sigma: float) -> float:
    """Third virial coefficient of the untruncated UF fluid, B3 = -1/3 int int f12 f13 f23,
    from the same expansion and the Gaussian integral
    int int exp(-a x^2 - b y^2 - c |x - y|^2) d^3x d^3y = (pi^2 / (ab + bc + ca))^(3/2):
    B3 = -(pi^3 sigma^6 / 3) sum_{k,l,m} c_k c_l c_m (kl + lm + mk)^(-3/2).  The alternating
    binomial sums cancel over many digits, so they are summed in 60-digit decimal arithmetic."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    cs = _uf_mayer_coefficients(p)
    s = Decimal(0)
    for k, ck in cs:
        for l, cl in cs:
            for m, cm in cs:
                q = Decimal(k * l + l * m + m * k)
                s += Decimal(ck * cl * cm) / (q * q.sqrt())
    return -(math.pi ** 3) * sigma ** 6 / 3.0 * float(s)


def ideal_gas_free_energy(n: int, volume: float, T: float, mass: float = M_SI) -> float:
    """Classical ideal gas of n identical atoms in volume V: F = -kB T ln(V^n / (n! Lambda^(3n)))
    with the thermal wavelength Lambda = hbar sqrt(2 pi / (m kB T)) (the end state of the
    switching that gives the UF fluid's free energy)."""
    kT = KB * T
    lam = HBAR * math.sqrt(2.0 * math.pi / (mass * MVV2E * kT))
    return -kT * (n * math.log(volume / lam ** 3) - math.lgamma(n + 1.0))



def einstein_free_energy(n: int, k: float, T: float, mass: float = M_SI) -> float:
    """Classical Einstein crystal, 3N independent oscillators of frequency sqrt(k/m):
    F = 3 N kB T ln(hbar omega / kB T).  The paper only says this F is known analytically
    (Sec. 2.1); the centre-of-mass correction is not applied (a reading)."""
    omega = math.sqrt(k / (mass * MVV2E))
    return 3.0 * n * KB * T * math.log(HBAR * omega / (KB * T))


def fl_lambda(tau):
    """Frenkel-Ladd switching function lambda(tau) = tau^5 (70 tau^4 - 315 tau^3 + 540 tau^2
    - 420 tau + 126), tau in [0, 1] (the schedule of the 64- and 8000-atom FL workloads)."""
    t = np.asarray(tau, dtype=np.float64)
    return t ** 5 * (70 * t ** 4 - 315 * t ** 3 + 540 * t ** 2 - 420 * t + 126)


def rs_lambda(tau, lam_f):
    """Reversible-scaling path lambda = 1 / (1 + tau (1/lambda_f - 1)) (Sec. 4, the LAMMPS
    variable ``lambda``), i.e. the physical temperature T0/lambda rises linearly in time."""
    t = np.asarray(tau, dtype=np.float64)
    return 1.0 / (1.0 + t * (1.0 / lam_f - 1.0))


def free_energy_difference(w_fwd, w_bwd):
    """Eq. dF: Delta F = (mean W_fwd - mean W_bwd) / 2."""
    return 0.5 * (np.mean(w_fwd) - np.mean(w_bwd))


def dissipated_heat(w_fwd, w_bwd):
    """Eq. Qdiss: Q = (mean W_fwd + mean W_bwd) / 2."""
    return 0.5 * (np.mean(w_fwd) + np.mean(w_bwd))


def helmholtz_from_switching(f_ref, w_fwd, w_bwd):
    """Eq. dA with the switching run going from the system of interest (lambda=0 here) to
    the reference (lambda=1): F_int = F_ref - (W_fwd - W_bwd)/2.  (The paper interpolates
    the other way round, lambda_i = 1 -> lambda_f = 0, which flips the sign of both works.)"""
    return f_ref - free_energy_difference(w_fwd, w_bwd)


def gibbs_from_helmholtz(f, p, v):
    """Eq. G_and_A: G = F + P V."""
    return f + p * v


def gibbs_rs(g0, n, T0, lam, w_fwd_to_lam, w_bwd_from_lam):
    """Eq. Gibbs_RS: G(P, T0/lambda) = G(P,T0)/lambda + 3/2 N kB T0 ln(lambda)/lambda
    + [W(1->lambda) - W(lambda->1)] / (2 lambda)."""
    lam = np.asarray(lam, dtype=np.float64)
    return (g0 / lam + 1.5 * n * KB * T0 * np.log(lam) / lam
            + (np.asarray(w_fwd_to_lam) - np.asarray(w_bwd_from_lam)) / (2.0 * lam))


def gibbs_as(g0, w_fwd, w_bwd):
    """Eq. Gibbs_AS: G(P,T) = G(P0,T) + [W(P0->P) - W(P->P0)] / 2."""
    return g0 + 0.5 * (np.asarray(w_fwd) - np.asarray(w_bwd))


def dcci_temp_update(ps_k, lam_k, lam_k1, du, dv):
    """Eq. Ps_coex_discreted: P_S(k+1) = P_S(k) - (lambda(k+1) - lambda(k)) dU/dV."""
    return ps_k - (lam_k1 - lam_k) * (du / dv)


def dcci_press_update(lam_k, p_k, p_k1, du, dv):
    """Eq. l_coex_discreted: lambda(k+1) = lambda(k) (1 + P_k dV/dU) / (1 + P_(k+1) dV/dU)."""
    return lam_k * (1.0 + p_k * dv / du) / (1.0 + p_k1 * dv / du)


# ------------------------------------------------------------------------------------------
# Time integration of one system, or of a coupled dCCI pair
# ------------------------------------------------------------------------------------------
SCHED_NONE, SCHED_FL, SCHED_RS, SCHED_AS = 0, 1, 2, 3
POT_SW, POT_EINSTEIN, POT_UF = 0, 1, 2
REF_EINSTEIN, REF_UF = 0, 1
BARO_NONE, BARO_ISO, BARO_ANISO = 0, 1, 2
DCCI_TEMP, DCCI_PRESS = 0, 1
DEGEN_DV = 1e-6      # A^3/atom: |dV| below this makes the temperature-control update singular
DEGEN_DU = 1e-12     # eV/atom: |dU| below this makes the pressure-control update singular


@dataclass
class System:
    """State and protocol of one simulated cell (all FP64, metal units, pressures in eV/A^3).

    Schedules (``sched``): NONE keeps lambda fixed; FL is the Hamiltonian interpolation
    H = K + (1-lambda) U_int + lambda U_E with U_E = k_E/2 sum |x - r0|^2, forward lambda
    0 -> 1 along ``fl_lambda``; RS is H = K + lambda U_int + lambda P V along ``rs_lambda``
    (forward 1 -> lambda_f); AS drives the barostat pressure linearly P0 -> P1 and its
    driving force is V.  ``direction`` = -1 runs FL/RS backward (tau -> 1 - tau).
    ``pot`` selects U_int: Stillinger-Weber, the Uhlenbeck-Ford fluid (parameters ``uf``), or
    (test mode) an Einstein crystal with spring ``k_int`` about r0 whose free energy is known in
    closed form (k_int = 0: no interaction, the ideal gas).  ``ref`` selects U_E of the FL
    interpolation: the Einstein crystal (springs k_E about r0) for solids, or the UF fluid for
    the liquid (Sec. 2.1: "for fluid-phase systems ... the Uhlenbeck-Ford model").
    """
    x: np.ndarray
    v: np.ndarray
    box: np.ndarray
    mass: float = M_SI
    dt: float = 0.001
    prm: tuple = SW_SI
    pot: int = POT_SW
    k_int: float = 0.0
    r0: np.ndarray | None = None
    k_E: float = 0.0
    T: float = 0.0
    tdamp: float = 0.0        # ps; <= 0: no thermostat (NVE)
    seed: int = 0
    sys_id: int = 0
    baro: int = BARO_NONE
    p_ext: float = 0.0        # eV/A^3 (physical P for RS; the barostat target is lambda P)
    pdamp: float = 1.0
    sched: int = SCHED_NONE
    direction: int = 1
    nsched: int = 1
    lam_f: float = 1.0        # RS
    p0: float = 0.0           # AS
    p1: float = 0.0           # AS
    lam: float = 1.0
    trace_every: int = 0
    ref: int = REF_EINSTEIN
    uf: tuple = (25.0, 2.0, 2200.0, 8.0)   # p, sigma (A), T_uf (K), rc (A)
    # dynamic state
    f: np.ndarray | None = None
    eta: np.ndarray = field(default_factory=lambda: np.zeros(3))
    k: int = 0
    W: float = 0.0
    p_tgt: float = 0.0
    u_int: float = 0.0
    u_ref: float = 0.0
    vir: np.ndarray = field(default_factory=lambda: np.zeros(6))
    kt: np.ndarray = field(default_factory=lambda: np.zeros(6))
    sums: np.ndarray = field(default_factory=lambda: np.zeros(5))   # H, dH/dl, P, V, count
    trace: list = field(default_factory=list)

    @property
    def n(self):
        return self.x.shape[0]

    # ---- protocol ---------------------------------------------------------------------
    def lam_at(self, k):
        tau = min(k / self.nsched, 1.0)
        if self.direction < 0:
            tau = 1.0 - tau
        if self.sched == SCHED_FL:
            return float(fl_lambda(tau))
        if self.sched == SCHED_RS:
            return float(rs_lambda(tau, self.lam_f))
        if self.sched == SCHED_AS:
            return self.p0 + (self.p1 - self.p0) * tau
        return self.lam

    def scales(self):
        """(scale of U_int forces, scale of U_E forces) at the current lambda."""
        if self.sched == SCHED_FL:
            return 1.0 - self.lam, self.lam
        if self.sched in (SCHED_RS,) or getattr(self, "_in_pair", False):
            return self.lam, 0.0
        return 1.0, 0.0

    def target_pressure(self):
        if self.sched == SCHED_RS:
            return self.lam * self.p_ext
        if self.sched == SCHED_AS:
            return self.lam
        return self.p_tgt if getattr(self, "_in_pair", False) else self.p_ext

    # ---- forces -----------------------------------------------------------------------
    def conservative_forces(self):
        """F = s_int F_int + s_E F_E at the current lambda; stores U_int, U_E, virial."""
        s_int, s_e = self.scales()
        f = np.zeros_like(self.x)
        if self.pot == POT_SW:
            e, fsw, vir, _ = sw_energy(self.x, self.box, self.prm)
            self.u_int = e
            self.vir = vir
            f += s_int * fsw
        elif self.pot == POT_UF:
            e, fuf, vir, _ = uf_energy(self.x, self.box, self.uf)
            self.u_int = e
            self.vir = vir
            f += s_int * fuf
        else:
            d = self.x - self.r0
            self.u_int = 0.5 * self.k_int * float(np.sum(d * d))
            self.vir = np.zeros(6)
            f += s_int * (-self.k_int * d)
        if self.sched == SCHED_FL and self.ref == REF_UF:
            e, fuf, _, _ = uf_energy(self.x, self.box, self.uf)
            self.u_ref = e
            f += s_e * fuf
        elif self.k_E > 0.0 and self.r0 is not None:
            d = self.x - self.r0
            self.u_ref = 0.5 * self.k_E * float(np.sum(d * d))
            f += s_e * (-self.k_E * d)
        else:
            self.u_ref = 0.0
        return f

    def langevin(self, v_half, step):
        """Damping -(m/tau) v plus sqrt(2 m kB T / (tau dt)) xi, with the per-system mean of
        the random part subtracted (the ``zero yes`` option the paper uses)."""
        if self.tdamp <= 0.0:
            return np.zeros_like(v_half)
        me = self.mass * MVV2E
        amp = math.sqrt(2.0 * me * KB * self.T / (self.tdamp * self.dt))
        xi = langevin_xi(self.seed, self.sys_id, step, self.n)
        xi = xi - xi.mean(axis=0)
        return -(me / self.tdamp) * v_half + amp * xi

    def kinetic_tensor(self):
        me = self.mass * MVV2E
        v = self.v
        return me * np.array([np.sum(v[:, 0] * v[:, 0]), np.sum(v[:, 1] * v[:, 1]),
                              np.sum(v[:, 2] * v[:, 2]), np.sum(v[:, 0] * v[:, 1]),
                              np.sum(v[:, 0] * v[:, 2]), np.sum(v[:, 1] * v[:, 2])])

    def volume(self):
        return float(self.box[0] * self.box[1] * self.box[2])

    def pressure_tensor(self):
        s_int, _ = self.scales()
        return (self.kt + s_int * self.vir) / self.volume()

    def setup(self):
        """Initial forces at step 0 (thermostat noise drawn with step counter 0)."""
        self.lam = self.lam_at(0) if self.sched != SCHED_NONE else self.lam
        if self.sched == SCHED_AS:
            self.p_tgt = self.lam
        self.f = self.conservative_forces() + self.langevin(self.v, 0)
        self.kt = self.kinetic_tensor()

    # ---- the two halves of a step (group update, then particle update) ----------------
    def observe(self):
        """Instantaneous P, V, driving force and Hamiltonian at the current step."""
        V = self.volume()
        Pt = self.pressure_tensor()
        P = float(Pt[:3].mean())
        K = 0.5 * float(self.kt[:3].sum())
        if self.sched == SCHED_FL:
            dhdl = self.u_ref - self.u_int                     # Eq. Wrev_HI integrand
            H = K + (1.0 - self.lam) * self.u_int + self.lam * self.u_ref
        elif self.sched == SCHED_RS:
            dhdl = self.u_int + self.p_ext * V                 # Eq. dH_RS with P_S = lambda P
            H = K + self.lam * self.u_int + self.lam * self.p_ext * V
        elif self.sched == SCHED_AS:
            dhdl = V                                           # Eq. Wmech integrand
            H = K + self.u_int + self.lam * V
        else:
            s_int, _ = self.scales()
            dhdl = 0.0
            H = K + s_int * self.u_int + (self.target_pressure() * V if self.baro else 0.0)
        return V, Pt, P, dhdl, H

    def barostat_kick(self, Pt):
        if self.baro == BARO_NONE:
            return
        V = self.volume()
        Qb = (self.n + 1) * KB * self.T * self.pdamp ** 2
        ptgt = self.target_pressure()
        if self.baro == BARO_ISO:
            g = 3.0 * V * (float(Pt[:3].mean()) - ptgt) / Qb
            self.eta = self.eta + self.dt * np.array([g, g, g])
        else:
            g = V * (Pt[:3] - ptgt) / Qb
            self.eta = self.eta + self.dt * g

    def particle_step(self):
        """Half kick, affine drift with the box, forces, Langevin, second half kick."""
        me = self.mass * MVV2E
        dt = self.dt
        v_half = self.v + (0.5 * dt / me) * self.f
        z = self.eta * dt
        s = np.exp(z)
        phi = np.where(z != 0.0, np.expm1(z) / np.where(z != 0.0, z, 1.0), 1.0)
        self.x = s * self.x + (dt * phi) * v_half
        self.box = self.box * s
        self.k += 1
        fc = self.conservative_forces()
        self.f = fc + self.langevin(v_half, self.k)
        self.v = v_half + (0.5 * dt / me) * self.f
        self.kt = self.kinetic_tensor()

    def record(self, V, P, dhdl, H):
        self.sums += np.array([H, dhdl, P, V, 1.0])
        if self.trace_every and self.k % self.trace_every == 0:
            self.trace.append((self.k, self.lam, self.W, dhdl, self.u_int, V, P, self.target_pressure(),
                               float(self.kt[:3].sum()) / ((3 * self.n - 3) * KB)))

    def step(self):
        V, Pt, P, dhdl, H = self.observe()
        self.record(V, P, dhdl, H)
        self.barostat_kick(Pt)
        if self.sched != SCHED_NONE:
            lam_next = self.lam_at(self.k + 1)
            self.W += dhdl * (lam_next - self.lam)             # Eq. Wdyn, left point
            self.lam = lam_next
        self.particle_step()

    def run(self, nsteps):
        if self.f is None:
            self.setup()
        for _ in range(nsteps):
            self.step()
        return self

    # ---- reporting ----------------------------------------------------------------------
    def temperature(self):
        return float(self.kt[:3].sum()) / ((3 * self.n - 3) * KB)

    def results(self):
        V, Pt, P, dhdl, H = self.observe()
        c = max(self.sums[4], 1.0)
        return dict(W=self.W, lam=self.lam, step=self.k, U=self.u_int, U_E=self.u_ref,
                    K=0.5 * float(self.kt[:3].sum()), T=self.temperature(), V=V,
                    P=Pt * EV_A3_TO_GPA, dHdl=dhdl, H=H, box=self.box.copy(),
                    mean_H=self.sums[0] / c, mean_dHdl=self.sums[1] / c,
                    mean_P=self.sums[2] / c * EV_A3_TO_GPA, mean_V=self.sums[3] / c)


class DcciPair:
    """Two systems (phase I, phase II) at fixed T0 whose common lambda and scaled pressure
    P_S follow the discrete dynamic Clausius-Clapeyron integration (Sec. 3).

    Temperature control (``mode`` TEMP): T(t) = T_i + (T_f - T_i) t/t_s, lambda = T0 / T(t)
    with T0 = T_i, and P_S by Eq. Ps_coex_discreted.  Pressure control (PRESS): P(t) =
    P_i + (P_f - P_i) t/t_s, lambda by Eq. l_coex_discreted and P_S = lambda P (Eq. P_sc).
    dU and dV are per-atom differences U_I/N_I - U_II/N_II, V_I/N_I - V_II/N_II (the CCE is
    written for molar quantities).  Coexistence estimates: T_coex = T0/lambda,
    P_coex = P_S/lambda.  The systems must use ``baro`` != NONE and ``sched`` NONE.
    """

    def __init__(self, s1: System, s2: System, T0, P0, mode, frm, to, nsteps):
        self.s = (s1, s2)
        self.T0, self.mode, self.frm, self.to, self.nsteps = T0, mode, frm, to, nsteps
        self.k = 0
        self.lam = 1.0
        self.ps = P0
        self.error = 0
        self.hist = []
        for s in self.s:
            s._in_pair = True
            s.lam = 1.0
            s.p_tgt = P0
            s.T = T0

    def control(self, k):
        tau = min(k / self.nsteps, 1.0)
        return self.frm + (self.to - self.frm) * tau

    def setup(self):
        for s in self.s:
            s.setup()

    def step(self):
        obs = [s.observe() for s in self.s]
        for s, (V, Pt, P, dhdl, H) in zip(self.s, obs):
            s.record(V, P, 0.0, H)
            s.barostat_kick(Pt)
        a, b = self.s
        du = a.u_int / a.n - b.u_int / b.n
        dv = obs[0][0] / a.n - obs[1][0] / b.n
        if self.mode == DCCI_TEMP:
            lam_next = self.control(0) / self.control(self.k + 1)   # T0 / T(t), T0 = T_i
            if abs(dv) < DEGEN_DV:
                self.error = 1
                lam_next, ps_next = self.lam, self.ps
            else:
                ps_next = dcci_temp_update(self.ps, self.lam, lam_next, du, dv)
        else:
            p_k, p_k1 = self.control(self.k), self.control(self.k + 1)
            if abs(du) < DEGEN_DU:
                self.error = 1
                lam_next, ps_next = self.lam, self.ps
            else:
                lam_next = dcci_press_update(self.lam, p_k, p_k1, du, dv)
                ps_next = lam_next * p_k1
        self.hist.append((self.k, self.lam, self.ps, du, dv))
        self.lam, self.ps = lam_next, ps_next
        self.k += 1
        for s in self.s:
            s.lam = self.lam
            s.p_tgt = self.ps
            s.particle_step()

    def run(self, nsteps):
        if self.s[0].f is None:
            self.setup()
        for _ in range(nsteps):
            self.step()
        return self

    def coexistence(self):
        return self.T0 / self.lam, self.ps / self.lam

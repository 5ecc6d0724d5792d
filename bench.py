#!/usr/bin/env python
"""Throughput benchmark: batched Frenkel-Ladd switching of 8000-atom diamond silicon.

Workload (per GPU): R replicas of an 8000-atom Si-cd crystal (10x10x10 cells, a = 5.431 A,
standard SW), Frenkel-Ladd switching to an Einstein crystal (k = 5 eV/A^2, lambda(tau) =
tau^5(70tau^4-315tau^3+540tau^2-420tau+126), 20000 steps per direction, half the replicas
forward and half backward) at 1000 K with a Langevin thermostat (0.1 ps), dt = 1 fs, FP32
pair/triplet arithmetic with FP64 positions, box, energies and work.  Inputs are synthetic
and seeded.  One timed step = one replay of the captured 32-MD-step graph over all
replicas (every MD step runs the whole path: group update, kick/drift, list rebuild when
the displacement test fires, forces with lambda mixing, Langevin, kick, work).

Prints one JSON line (see the keys below).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (batched FP32/FP64 vs plain FP64, 1 GB300), % HBM roofline, ΔG err"
UNIT = "atom-steps/s"
KB = 8.617333262e-5
MVV2E = 1.66053906660e-23 / 1.602176634e-19
MASS = 28.0855
NCELL = 10          # 10x10x10 diamond cells = 8000 atoms
T_SW = 1000.0
K_E = 5.0
NSCHED = 20000
MD_STEPS = 32       # MD steps per timed step (one graph replay)
SKIN = 0.7          # Verlet skin (A) of the dCCI, reversible-scaling and comparator contexts
FL_SKIN = 1.6       # Verlet skin (A) of the timed Frenkel-Ladd crystal: with rcs = 5.37 A the rows hold the
                    # first three neighbour shells (28 entries; the fourth lies at 5.43 A), and an atom of
                    # the 1000 K crystal rarely moves skin/2 = 0.8 A, so lists are almost never rebuilt
                    # (measured 0.7 / 1.0 / 1.2 / 1.4 / 1.6 A); lists are exact at any skin
# Algorithmic bytes per atom of the two force passes (FP32 path, Frenkel-Ladd), m = mean
# in-cutoff shell size, nbar = mean Verlet row length:
#   pass A (edges): own mirror 16 + row length 4 + row 4 nbar + shell indices 4 m + leg forces
#                   16 m + shell size 4 + partial force and energy 16;
#   pass B (gather): partial force 16 + shell size 4 + own shell indices 4 m + the neighbours'
#                    leg forces 16 m + spring offset 16 + displacement 24 + noise 16 + v read 12
#                    + v write 12 + total force write 16.
# Whole step (the method's minimum, FP64 x and v, r0, F, list): 212 B per atom-step.
PASS_A_FIXED = 16 + 4 + 4 + 16
PASS_B_FIXED = 16 + 4 + 16 + 24 + 16 + 12 + 12 + 16
STEP_BYTES = 212.0


def workload_config(replicas, skin=SKIN):
    return {"workload": f"Frenkel-Ladd switching, {replicas} x 8000-atom Si-cd (SW), 1000 K, k=5 eV/A^2",
            "atoms_per_replica": 8 * NCELL ** 3, "replicas_per_gpu": replicas,
            "md_steps_per_step": MD_STEPS, "dt_fs": 1.0, "switch_steps": NSCHED,
            "timed_window": "after the untimed equilibration and warm-up steps of the switching run",
            "l2": "inputs larger than L2 (no flush)", "verlet_skin_A": skin}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    """Hash of the kernel source's code: comments and blank lines are left out, so an edit of the
    comments alone does not retire a traffic record taken on the same code."""
    with open(os.path.join(ROOT, "paper_2103_10449_gb300", "csrc", "nefe_kernels.cu")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [ln.split("//", 1)[0].rstrip() for ln in src.splitlines()]
    code = "\n".join(ln for ln in lines if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per atom of `kernel` from the committed ncu summary, if that summary was taken
    on the current kernel source and for this kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "force_passes_traffic.txt")
    try:
        txt = open(path).read()
    except OSError:
        return None
    k = re.search(r"^kernel:\s*(\w+)", txt, re.M)
    m = re.search(r"kernel_source_sha256_16:\s*(\w+)", txt)
    b = re.search(r"dram_bytes_per_atom:\s*([0-9.eE+-]+)", txt)
    if not k or not m or not b or k.group(1) != kernel or m.group(1) != kernel_hash():
        return None
    return float(b.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_context(N, replicas, precision, seed0=1000, stream=None, skin=None, first=0):
    """Replicas first .. first + replicas - 1 of the benchmark workload (replica u: seed seed0 + u,
    forward when u is even, backward when odd), so a sharded job holds the same set of replicas
    whatever the number of ranks."""
    from paper_2103_10449_gb300 import inputs as I
    x, box = I.diamond(NCELL, NCELL, NCELL)
    sv = math.sqrt(KB * T_SW / (MASS * MVV2E))
    ctx = N.Context(precision=precision, dt=0.001, skin=SKIN if skin is None else skin, nbr_cap=48, stream=stream)
    for u in range(first, first + replicas):
        v = I.gaussian_velocities(len(x), sv, seed0 + u)
        s = ctx.add_system(x, box, v=v, r0=x, mass=MASS)
        ctx.set_thermostat(s, T_SW, 0.1, seed0 + u)
        ctx.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if u % 2 == 0 else -1, nsteps=NSCHED, k_E=K_E)
    ctx.setup()
    return ctx, len(x)


class FLEngine:
    """One rank's replicas [lo, hi) of the Frenkel-Ladd benchmark workload, driven by
    sharding.run_sharded: equilibrated, autotuned (or fixed lanes), profiled."""

    def __init__(self, N, torch, lo, hi, args):
        self.N, self.torch = N, torch
        self.stream = torch.cuda.Stream()
        self.lo, self.hi = lo, hi
        self.ctx, self.natoms = build_context(N, hi - lo, N.NEFE_FP32, stream=self.stream, skin=args.skin, first=lo)
        self.ctx.run(args.equil)
        if args.tuning:
            t = [int(v) for v in args.tuning.split(",")]
            self.ctx.set_tuning(t[0], t[1])
            if len(t) > 2:
                self.ctx.set_rebuild_policy(t[2])
        else:
            self.ctx.autotune()

    def warmup(self, k):
        for _ in range(k):
            self.ctx.run(MD_STEPS)
        self.ctx.sync()
        self.launches0 = self.ctx.launch_count()

    def timed(self, k):
        return time_steps(self.torch, self.ctx, self.stream, k, MD_STEPS)

    def rows(self):
        return [(self.lo + j, r["W"], r["lambda"], int(r["error"])) for j, r in enumerate(self.ctx.results_all())]


class DcciEngine:
    """One rank's pairs [lo, hi) of the batched dCCI workload (64 Si-cd / beta-Sn pairs of
    log-uniform size), driven by sharding.run_sharded."""

    def __init__(self, N, torch, lo, hi, sizes):
        from paper_2103_10449_gb300 import inputs as I
        self.N, self.torch = N, torch
        self.stream = torch.cuda.Stream()
        sv = math.sqrt(KB * 400.0 / (MASS * MVV2E))
        self.ctx = N.Context(precision=N.NEFE_FP32, dt=0.001, skin=SKIN, nbr_cap=48, stream=self.stream)
        self.pairs = []
        self.lo = lo
        for k in range(lo, hi):
            n = sizes[k]
            xa, ba = I.diamond(*I.diamond_cells_for(n))
            xb, bb = I.beta_tin(*I.beta_tin_cells_for(n))
            a = self.ctx.add_system(xa, ba, v=I.gaussian_velocities(len(xa), sv, 3000 + 2 * k), mass=MASS)
            b = self.ctx.add_system(xb, bb, v=I.gaussian_velocities(len(xb), sv, 3001 + 2 * k), mass=MASS)
            for sidx, seed in ((a, 3000 + 2 * k), (b, 3001 + 2 * k)):
                self.ctx.set_thermostat(sidx, 400.0, 0.1, seed)
            self.ctx.set_barostat(a, N.NEFE_BARO_ISO, 10.0, 0.5)
            self.ctx.set_barostat(b, N.NEFE_BARO_ANISO, 10.0, 0.5)
            self.pairs.append(self.ctx.pair_dcci(a, b, 400.0, 10.0, N.NEFE_DCCI_PRESS, 10.0, 15.0, 100000))
        self.ctx.setup()
        self.ctx.run(320)
        self.ctx.autotune()

    def warmup(self, k):
        self.ctx.run(k * MD_STEPS)
        self.ctx.sync()

    def timed(self, k):
        return time_steps(self.torch, self.ctx, self.stream, k, MD_STEPS)

    def rows(self):
        out = []
        for j, p in enumerate(self.pairs):
            T, P, lam, err = self.ctx.pair(p)
            out.append((self.lo + j, T, P, int(err)))
        return out


def dcci_pair_atoms(sizes):
    from paper_2103_10449_gb300 import inputs as I
    out = []
    for n in sizes:
        nx, ny, nz = I.diamond_cells_for(n)
        mx, my, mz = I.beta_tin_cells_for(n)
        out.append(8 * nx * ny * nz + 4 * mx * my * mz)
    return out


def free_energy_error(N, reps=8, n_eq=500, n_sw=2000):
    """FP32 against FP64 free-energy estimate of the same switching experiment.

    reps forward (SW -> Einstein) and reps backward (Einstein -> SW) Frenkel-Ladd realisations
    of the 8000-atom crystal at 1000 K, n_sw steps each, from endpoint states equilibrated for
    n_eq steps in FP64; both precisions start from identical states with identical noise
    seeds.  Returns the switching part of the free energy, -1/2 (<W_f> - <W_b>)/N (the
    Einstein reference term is the same for both and cancels in the error), per precision,
    their difference and the standard error of the estimate itself."""
    from paper_2103_10449_gb300 import inputs as I
    x, box = I.diamond(NCELL, NCELL, NCELL)
    n = len(x)
    sv = math.sqrt(KB * T_SW / (MASS * MVV2E))
    eq = N.Context(precision=N.NEFE_FP64, dt=0.001, skin=0.5, nbr_cap=48)
    for r in range(2 * reps):
        fwd = r < reps
        s = eq.add_system(x, box, v=I.gaussian_velocities(n, sv, 5000 + r), r0=x, mass=MASS,
                          pot=N.NEFE_POT_SW if fwd else N.NEFE_POT_EINSTEIN, k_int=0.0 if fwd else K_E)
        eq.set_thermostat(s, T_SW, 0.1, 5000 + r)
    eq.run(n_eq)
    states = [eq.get_state(r)[:2] for r in range(2 * reps)]
    eq.close()
    out = {}
    for name, prec in (("fp64", N.NEFE_FP64), ("fp32", N.NEFE_FP32)):
        c = N.Context(precision=prec, dt=0.001, skin=SKIN, nbr_cap=48)
        for r in range(2 * reps):
            s = c.add_system(states[r][0], box, v=states[r][1], r0=x, mass=MASS)
            c.set_thermostat(s, T_SW, 0.1, 7000 + r)
            c.set_schedule(s, N.NEFE_SCHED_FL, direction=1 if r < reps else -1, nsteps=n_sw, k_E=K_E)
        c.run(n_sw)
        res = c.results_all()
        c.close()
        wf = np.array([res[r]["W"] for r in range(reps)])
        wb = np.array([res[r]["W"] for r in range(reps, 2 * reps)])
        out[name] = (-0.5 * (wf.mean() - wb.mean()) / n,
                     0.5 * math.sqrt(wf.var(ddof=1) / reps + wb.var(ddof=1) / reps) / n,
                     sum(int(r["error"] != 0) for r in res))
    return {"dF_switch_fp64_eV_per_atom": out["fp64"][0], "dF_switch_fp32_eV_per_atom": out["fp32"][0],
            "dG_err_meV_per_atom": 1000.0 * (out["fp32"][0] - out["fp64"][0]),
            "stat_err_meV_per_atom": 1000.0 * out["fp64"][1],
            "protocol": f"{reps} forward + {reps} backward FL realisations, {n_sw} steps each, 8000 atoms, 1000 K,"
                        f" identical initial states and noise seeds in both precisions",
            "systems_with_errors": out["fp64"][2] + out["fp32"][2]}


def precision_errors(N, reps=4, n_eq=2000, n_dcci=10000, n_rs=5000):
    """FP32 against FP64 for the other results of the path, each from identical initial states
    (equilibrated in FP64) with identical noise seeds in both precisions:
    * the dCCI coexistence pressure: reps Si-cd (8000 atoms) / beta-Sn (8000 atoms) pairs in
      temperature control from (400 K, 13.09 GPa) to 600 K over n_dcci steps, P_coex at the end;
    * the reversible-scaling work: reps Si-cd replicas at 10 GPa, lambda 1 -> 0.5 over n_rs steps.
    Returns each estimate per precision, their difference and the statistical error of the
    FP64 estimate (standard error over the realisations)."""
    from paper_2103_10449_gb300 import inputs as I
    T0, P0, P_rs = 400.0, 13.09, 10.0
    xa, ba = I.diamond(NCELL, NCELL, NCELL)
    xb, bb = I.beta_tin(*I.beta_tin_cells_for(8000))
    sv = math.sqrt(KB * T0 / (MASS * MVV2E))
    eq = N.Context(precision=N.NEFE_FP64, dt=0.001, skin=SKIN, nbr_cap=48)
    for r in range(reps):
        for k, (x, b, mode) in enumerate(((xa, ba * 0.96, N.NEFE_BARO_ISO), (xb, bb, N.NEFE_BARO_ANISO))):
            s = eq.add_system(x * (b[0] / (ba[0] if k == 0 else bb[0])), b,
                              v=I.gaussian_velocities(len(x), sv, 8000 + 2 * r + k))
            eq.set_thermostat(s, T0, 0.1, 8000 + 2 * r + k)
            eq.set_barostat(s, mode, P0, 1.0)
    for r in range(reps):
        s = eq.add_system(xa * 0.98, ba * 0.98, v=I.gaussian_velocities(len(xa), sv, 8100 + r))
        eq.set_thermostat(s, T0, 0.1, 8100 + r)
        eq.set_barostat(s, N.NEFE_BARO_ISO, P_rs, 1.0)
    eq.run(n_eq)
    st = [eq.get_state(s) for s in range(3 * reps)]
    eq.close()
    out = {}
    for name, prec in (("fp64", N.NEFE_FP64), ("fp32", N.NEFE_FP32)):
        c = N.Context(precision=prec, dt=0.001, skin=SKIN, nbr_cap=48)
        pids = []
        for r in range(reps):
            a = c.add_system(st[2 * r][0], st[2 * r][2], v=st[2 * r][1])
            b = c.add_system(st[2 * r + 1][0], st[2 * r + 1][2], v=st[2 * r + 1][1])
            c.set_thermostat(a, T0, 0.1, 8200 + 2 * r)
            c.set_thermostat(b, T0, 0.1, 8201 + 2 * r)
            c.set_barostat(a, N.NEFE_BARO_ISO, P0, 1.0)
            c.set_barostat(b, N.NEFE_BARO_ANISO, P0, 1.0)
            pids.append(c.pair_dcci(a, b, T0, P0, N.NEFE_DCCI_TEMP, T0, 600.0, n_dcci))
        rs = []
        for r in range(reps):
            x, v, b = st[2 * reps + r]
            s = c.add_system(x, b, v=v)
            c.set_thermostat(s, T0, 0.1, 8300 + r)
            c.set_barostat(s, N.NEFE_BARO_ISO, P_rs, 1.0)
            c.set_schedule(s, N.NEFE_SCHED_RS, nsteps=n_rs, lambda_f=0.5, P_GPa=P_rs)
            rs.append(s)
        # pressure switching of both solids from 13.09 to 14 GPa at 400 K (the step that fixes the
        # 400 K coexistence pressure): the switching work per atom of each phase
        asw = []
        for r in range(reps):
            for k, mode in ((0, N.NEFE_BARO_ISO), (1, N.NEFE_BARO_ANISO)):
                x, v, b = st[2 * r + k]
                s = c.add_system(x, b, v=v)
                c.set_thermostat(s, T0, 0.1, 8400 + 2 * r + k)
                c.set_barostat(s, mode, P0, 1.0)
                c.set_schedule(s, N.NEFE_SCHED_AS, nsteps=n_rs, P0_GPa=P0, P1_GPa=14.0)
                asw.append(s)
        c.run(n_rs)
        w = np.array([c.results(s)["W"] / len(xa) for s in rs])
        w_as = np.array([c.results(s)["W"] / (len(xa) if j % 2 == 0 else len(xb)) for j, s in enumerate(asw)])
        v_as = np.array([c.results(s)["V"] / (len(xa) if j % 2 == 0 else len(xb)) for j, s in enumerate(asw)])
        c.run(n_dcci - n_rs)
        pc = np.array([c.pair(p)[1] for p in pids])
        errs = sum(int(r["error"] != 0) for r in c.results_all())
        c.close()
        out[name] = (pc, w, errs, w_as, v_as)
    p64, w64, e64, a64, v64 = out["fp64"]
    p32, w32, e32, a32, _ = out["fp32"]
    # the coexistence pressure moves by the error of G_cd - G_beta-tin over the volume difference
    d_as = (a32[0::2] - a64[0::2]).mean() - (a32[1::2] - a64[1::2]).mean()
    dv = v64[0::2].mean() - v64[1::2].mean()
    return {"dcci_P_coex": {"fp64_GPa": float(p64.mean()), "fp32_GPa": float(p32.mean()),
                            "err_GPa": float(p32.mean() - p64.mean()),
                            "stat_err_GPa": float(p64.std(ddof=1) / math.sqrt(reps)),
                            "protocol": f"{reps} Si-cd/beta-Sn pairs (8000 + 8000 atoms), temperature control "
                                        f"400 -> 600 K over {n_dcci} steps from 13.09 GPa"},
            "as_W": {"cd_err_meV_per_atom": float(1000.0 * (a32[0::2] - a64[0::2]).mean()),
                     "betasn_err_meV_per_atom": float(1000.0 * (a32[1::2] - a64[1::2]).mean()),
                     "implied_P_coex_err_GPa": float(d_as / dv * 160.21766340),
                     "protocol": f"{reps} Si-cd and {reps} beta-Sn replicas, pressure switching 13.09 -> 14 GPa at "
                                 f"400 K over {n_rs} steps; P_coex error = error of (G_cd - G_beta-Sn) / dV"},
            "rs_W": {"fp64_eV_per_atom": float(w64.mean()), "fp32_eV_per_atom": float(w32.mean()),
                     "err_meV_per_atom": float(1000.0 * (w32.mean() - w64.mean())),
                     "stat_err_meV_per_atom": float(1000.0 * w64.std(ddof=1) / math.sqrt(reps)),
                     "protocol": f"{reps} Si-cd replicas (8000 atoms) at 10 GPa, lambda 1 -> 0.5 over {n_rs} steps"},
            "systems_with_errors": e64 + e32}


def differentiation_throughput(N, torch):
    """The differentiation workload: (i) the SW energy + forces + seven parameter derivatives
    (nefe_sw_energy_grad, the backward of the autograd.Function) on diamond cells from 8000 to
    1,000,000 atoms, atoms/s per precision; (ii) the checkpointed adjoint of the switching work
    over 2000 steps of a 32768-atom liquid at 1700 K (K_c = 45), atom-steps/s of the forward
    run and of the reverse sweep (which recomputes every segment)."""
    from paper_2103_10449_gb300 import inputs as I
    out = {"grad_sweep_atoms_per_s": {}}
    prm = N.nefe_sw_params_silicon()
    rcs = 1.80 * 2.0951 + 0.5
    cap = 48
    for nc in (10, 20, 32, 40, 50):
        x, box = I.diamond(nc, nc, nc)
        n = len(x)
        xd = torch.tensor(np.ascontiguousarray(x.T).reshape(-1), dtype=torch.float64, device="cuda")
        nbr = torch.empty(n * cap, dtype=torch.int32, device="cuda")
        cnt = torch.empty(n, dtype=torch.int32, device="cuda")
        f = torch.empty(3 * n, dtype=torch.float64, device="cuda")
        eg = torch.empty(8, dtype=torch.float64, device="cuda")
        N.nefe_neighbor_build(xd, n, box, rcs, cap, nbr, cnt)
        row = {}
        grads = {}
        for name, prec in (("fp32", N.NEFE_FP32), ("fp64", N.NEFE_FP64)):
            for _ in range(2):
                N.nefe_sw_energy_grad(xd, n, box, rcs, nbr, cnt, cap, prm, prec, f, eg)
            torch.cuda.synchronize()
            grads[name] = eg.cpu().numpy().copy()
            reps = 5
            t0 = time.perf_counter()
            for _ in range(reps):
                N.nefe_sw_energy_grad(xd, n, box, rcs, nbr, cnt, cap, prm, prec, f, eg)
            torch.cuda.synchronize()
            row[name] = n * reps / (time.perf_counter() - t0)
        out["grad_sweep_atoms_per_s"][str(n)] = row
        g32, g64 = grads["fp32"], grads["fp64"]
        out.setdefault("dE_dtheta_fp32_rel_err", {})[str(n)] = float(
            np.max(np.abs(g32[1:] - g64[1:])) / np.max(np.abs(g64[1:])))
        del xd, nbr, cnt, f
    x, box = I.liquid(32768, 0.05425, seed=51)
    v = I.gaussian_velocities(len(x), math.sqrt(KB * 1700.0 / (MASS * MVV2E)), 52)
    ctx = N.Context(precision=N.NEFE_FP32)
    s = ctx.add_system(x, box, v=v)
    ctx.set_thermostat(s, 1700.0, 0.1, 53)
    ctx.run(1000)
    x0, v0, _ = ctx.get_state(s)
    ctx.close()
    adj = N.Adjoint(x0, v0, box, kind=N.NEFE_SCHED_RS, lambda_f=0.5, T=1700.0, tdamp=0.1, seed=54, nsched=2000,
                    checkpoint_every=45)
    K = 2000
    t0 = time.perf_counter()
    adj.forward(K)
    t1 = time.perf_counter()
    g = adj.backward()
    t2 = time.perf_counter()
    adj.close()
    out["adjoint"] = {"workload": "32768-atom liquid Si, 1700 K, reversible scaling 1 -> 0.5, 2000 steps, K_c = 45, FP64",
                      "forward_atom_steps_per_s": len(x0) * K / (t1 - t0),
                      "backward_atom_steps_per_s": len(x0) * K / (t2 - t1),
                      "dW_dtheta": [float(v) for v in g]}
    return out


def dcci_batched_throughput(N, torch, pairs=64, steps=5, rank=0, world=1, dist=None, barrier=None):
    """The batched dCCI workload: `pairs` coupled Si-cd / beta-Sn pairs of uneven sizes
    (log-uniform 512..32768 atoms per phase, from a fixed seed), pressure-controlled coexistence
    integration from 10 GPa at 400 K (Eq. l_coex_discreted), FP32 kernels, captured graph;
    atom-steps/s over `steps` graph replays after equilibration and autotuning.  With several
    ranks each takes a contiguous range of pairs balanced by atom count (a pair never splits:
    its two phases exchange U and V every step) and the coexistence estimates of all pairs are
    gathered at the end."""
    from paper_2103_10449_gb300 import inputs as I
    from paper_2103_10449_gb300 import sharding as SH
    sizes = I.log_uniform_sizes(pairs, 512, 32768, seed=2021)
    atoms = dcci_pair_atoms(sizes)
    out = SH.run_sharded(atoms, rank, world, lambda lo, hi: DcciEngine(N, torch, lo, hi, sizes), 2, steps,
                         MD_STEPS, dist=dist, device=torch.device("cuda", torch.cuda.current_device()),
                         barrier=barrier)
    errors = sum(1 for r in out["rows"] if r[3] != 0)
    out["engine"].ctx.close()
    return {"workload": f"{pairs} Si-cd/beta-Sn dCCI pairs, 512..32768 atoms per phase (log-uniform), "
                        f"pressure control 10 -> 15 GPa at 400 K, FP32 kernels",
            "atoms": int(sum(atoms)), "atom_steps_per_s": out["value"], "ranks": world,
            "pairs_per_rank": [list(r) for r in SH.shard_units(atoms, world)],
            "pairs_gathered": len(out["rows"]), "pairs_with_errors": errors}


def rs_npt_batched_throughput(N, torch, per_phase=20, steps=5):
    """The reversible-scaling NPT workload: Si-cd (8000 atoms), beta-Sn (8192) and liquid (8000,
    random positions at 2.53 g/cm^3) at 0 and 10 GPa, `per_phase` replicas of each phase and
    pressure in one context (lambda 1 -> 0.2, i.e. 400 -> 2000 K, over 50000 steps; isotropic
    barostat for cd and liquid, anisotropic for beta-Sn), FP32 kernels; atom-steps/s."""
    from paper_2103_10449_gb300 import inputs as I
    sv = math.sqrt(KB * 400.0 / (MASS * MVV2E))
    stream = torch.cuda.Stream()
    ctx = N.Context(precision=N.NEFE_FP32, dt=0.001, skin=SKIN, nbr_cap=48, stream=stream)
    cd = I.diamond(10, 10, 10)
    bt = I.beta_tin(8, 16, 16)
    lq = I.liquid(8000, 0.05425, seed=4242)
    natoms = 0
    k = 0
    for P in (0.0, 10.0):
        for (x, box), baro in ((cd, N.NEFE_BARO_ISO), (bt, N.NEFE_BARO_ANISO), (lq, N.NEFE_BARO_ISO)):
            for r in range(per_phase):
                s = ctx.add_system(x, box, v=I.gaussian_velocities(len(x), sv, 6000 + k), mass=MASS)
                ctx.set_thermostat(s, 400.0, 0.1, 6000 + k)
                ctx.set_barostat(s, baro, P, 1.0)
                ctx.set_schedule(s, N.NEFE_SCHED_RS, nsteps=50000, lambda_f=0.2, P_GPa=P)
                natoms += len(x)
                k += 1
    ctx.setup()
    ctx.run(320)
    ctx.autotune()
    ctx.run(2 * MD_STEPS)
    ctx.sync()
    wall = time_steps(torch, ctx, stream, steps, MD_STEPS)
    errors = sum(1 for r in ctx.results_all() if r["error"] != 0)
    ctx.close()
    return {"workload": f"reversible scaling NPT, {per_phase} replicas each of 8000-atom Si-cd, 8192-atom beta-Sn "
                        f"and 8000-atom liquid at 0 and 10 GPa (lambda 1 -> 0.2 over 50000 steps), FP32 kernels",
            "atoms": natoms, "atom_steps_per_s": natoms * MD_STEPS * steps / wall, "systems_with_errors": errors}


def time_steps(torch, ctx, stream, steps, md_steps):
    """Seconds for `steps` timed steps, from CUDA events on the context's stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        ctx.run(md_steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1000.0


def cpu_baseline_sample(target_s=15.0):
    """The FP64 oracle, as it stands, on one 8000-atom replica of the workload (single thread)."""
    from oracle import oracle as O
    from paper_2103_10449_gb300 import inputs as I
    x, box = I.diamond(NCELL, NCELL, NCELL)
    v = I.gaussian_velocities(len(x), math.sqrt(O.KB * T_SW / (O.M_SI * O.MVV2E)), 1000)
    s = O.System(x=x.copy(), v=v, box=box.copy(), r0=x.copy(), k_E=K_E, T=T_SW, tdamp=0.1, seed=1000,
                 sched=O.SCHED_FL, nsched=NSCHED)
    s.setup()
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < target_s or n < 2:
        s.step()
        n += 1
    dt = time.perf_counter() - t0
    return len(x) * n / dt, n, dt


def run_reference(args, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2103_10449_gb300 import inputs as I
    O.build()
    x, box = I.diamond(NCELL, NCELL, NCELL)
    v = I.gaussian_velocities(len(x), math.sqrt(O.KB * T_SW / (O.M_SI * O.MVV2E)), 1000)
    s = O.System(x=x.copy(), v=v, box=box.copy(), r0=x.copy(), k_E=K_E, T=T_SW, tdamp=0.1, seed=1000,
                 sched=O.SCHED_FL, nsched=NSCHED)
    s.setup()
    per_step = 2     # oracle MD steps per timed step (bounded sample of the workload)
    for _ in range(args.warmup):
        for _ in range(per_step):
            s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(per_step):
            s.step()
    dt = time.perf_counter() - t0
    value = len(x) * per_step * args.steps / dt
    sample = f"{per_step} MD steps of one 8000-atom replica per timed step (O(N^2) FP64 oracle)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.replicas),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "host_cores_available": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def spawn_ranks(args):
    """`--gpus N` without a launcher: start N ranks (one process per GPU) through torch's launcher,
    exactly as a torchrun launch would; rank 0 prints the JSON line."""
    import socket
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nefe", choices=["nefe", "reference"])
    ap.add_argument("--replicas", type=int, default=128, help="replicas per GPU")
    ap.add_argument("--equil", type=int, default=3000,
                    help="untimed MD steps before warm-up (thermalises the crystals)")
    ap.add_argument("--no-extras", action="store_true", help="skip comparators, e2e and CPU baseline")
    ap.add_argument("--skin", type=float, default=FL_SKIN, help="Verlet skin (A) of the timed context")
    ap.add_argument("--tuning", default=None,
                    help="pass A,pass B lanes per atom[,rebuild policy] instead of autotuning (e.g. to profile a chosen "
                         "configuration)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    if "WORLD_SIZE" not in os.environ and args.gpus > 1 and args.impl == "nefe":
        sys.exit(spawn_ranks(args))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    dist = None
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2103_10449_gb300 import nefe as N
    from paper_2103_10449_gb300 import sharding as SH
    N.load()
    R = args.replicas
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # the whole job: world x R replicas, each rank takes its contiguous share (weak scaling)
    clocks = ClockSampler(local)

    def clocks_start():
        clocks.start()
        time.sleep(0.3)

    run = SH.run_sharded([8 * NCELL ** 3] * (world * R), rank, world, lambda lo, hi: FLEngine(N, torch, lo, hi, args),
                         args.warmup, args.steps, MD_STEPS, dist=dist, device=dev, barrier=barrier,
                         before_timed=clocks_start, after_timed=None)
    clk = clocks.stop()
    eng = run["engine"]
    ctx = eng.ctx
    natoms = eng.natoms
    wall = run["wall_max"]
    value = run["value"]
    launches = ctx.launch_count() - eng.launches0
    # per-pass CUDA-event durations: one graph replay with events around the force passes, after
    # the timed region (the timed graph carries no event nodes)
    ctx.set_profiling(True)
    ctx.run(MD_STEPS)
    a_us, b_us, nsamp = ctx.profile()
    ctx.set_profiling(False)
    mean_cnt, max_cnt, nbuild = ctx.list_stats(-1)
    errors = sum(1 for r in run["rows"] if r[3] != 0)
    atoms = natoms * (run["range"][1] - run["range"][0])

    # roofline of the dominant kernel (the longer force pass), from live CUDA-event durations
    m_shell, _ = ctx.shell_stats()
    lanes = list(ctx.lanes())
    bytes_a = PASS_A_FIXED + 4.0 * mean_cnt + 20.0 * m_shell
    bytes_b = PASS_B_FIXED + 20.0 * m_shell
    if lanes[0] == 0:
        # scatter form: pass A reads own mirror, row length and row, and adds the leg forces into
        # 16-byte accumulators (L2-resident reductions, not counted); pass B streams the
        # epilogue operands (accumulator 16, spring offset 16, displacement 24, noise 16, v 12 +
        # 12, force 16)
        bytes_a = 16 + 4 + 4.0 * mean_cnt + 4
        bytes_b = 16 + 16 + 24 + 16 + 12 + 12 + 16
    if b_us > a_us:
        kkey, kname, kbytes, kus = "k_gather", "force pass B (gather or scatter-form epilogue: springs, Langevin, kick)", bytes_b, b_us
    else:
        kkey, kname, kbytes, kus = "k_edges", "force pass A (shell, pair terms, triplet leg forces)", bytes_a, a_us
    achieved = kbytes * atoms / (kus * 1e-6) / 1e9
    peak, peak_kind = peaks()
    tr = recorded_traffic(kkey)
    step_gbs = value / world * STEP_BYTES / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None if tr is None else tr * atoms,
                "kernel": kname, "algorithmic_bytes_per_atom": kbytes, "kernel_us_mean": kus,
                "pass_a_us_mean": a_us, "pass_b_us_mean": b_us,
                "step_achieved_gbs": step_gbs, "step_frac": step_gbs / peak,
                "step_bytes_per_atom_step": STEP_BYTES,
                "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "lanes_per_atom": lanes[0],
                "lanes_pass_a_pass_b_list": lanes, "rebuild_all_systems": ctx.rebuild_policy()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(R, args.skin), "roofline": roofline, "clocks": clk, "gpu_launches": launches,
            "list": {"mean_row": mean_cnt, "max_row": max_cnt, "builds": nbuild, "mean_shell": m_shell},
            "systems_with_errors": errors,
            "sharding": {"ranks": world, "replicas_per_rank": R, "replicas_gathered": len(run["rows"]),
                         "collectives": "max of the timed interval, all-gather of per-replica results (after the timed region)"}}
    ctx.close()
    del eng

    if not args.no_extras and world > 1:
        # several ranks: the batched dCCI workload sharded over all ranks (pairs by atom count)
        line["dcci_batched"] = dcci_batched_throughput(N, torch, rank=rank, world=world, dist=dist, barrier=barrier)
    if not args.no_extras and world == 1:
        # e2e through the public API with host buffers: upload state, run, read results
        ctx, _ = build_context(N, R, N.NEFE_FP32, seed0=1000)
        ntot = natoms * R
        xh = torch.empty((ntot, 3), dtype=torch.float64, pin_memory=True).numpy()
        vh = torch.empty((ntot, 3), dtype=torch.float64, pin_memory=True).numpy()
        ctx.get_state_all(xh, vh)
        for _ in range(2):
            ctx.set_state_all(xh, vh); ctx.run(MD_STEPS); ctx.results_all()
        e_steps = max(3, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            ctx.set_state_all(xh, vh)
            ctx.run(MD_STEPS)
            ctx.results_all()
        e2e_wall = time.perf_counter() - t0
        line["e2e"] = {"value": ntot * MD_STEPS * e_steps / e2e_wall, "unit": UNIT,
                       "h2d_bytes_per_step": 2 * 8 * 3 * ntot,
                       "d2h_bytes_per_step": R * 8 * 32,
                       "path": "nefe_set_state_all (pinned host x, v) + nefe_run + nefe_get_results_all"}
        del ctx
        # comparators on the same GPU: plain FP64 single replica, FP32 single replica, FP64 batched
        comp = {}
        for name, reps, prec, steps, eq in (("fp64_single_replica", 1, N.NEFE_FP64, 20, 1000),
                                            ("fp32_single_replica", 1, N.NEFE_FP32, 20, 1000),
                                            ("fp64_batched", R, N.NEFE_FP64, 3, 200)):
            s2 = torch.cuda.Stream()
            c2, na = build_context(N, reps, prec, stream=s2, skin=args.skin)   # same list radius
            c2.run(eq)
            c2.autotune()
            for _ in range(2):
                c2.run(MD_STEPS)
            c2.sync()
            w = time_steps(torch, c2, s2, steps, MD_STEPS)
            comp[name] = na * reps * MD_STEPS * steps / w
            del c2
        comp["batched_fp32_over_fp64_single"] = value / world / comp["fp64_single_replica"]
        comp["batched_fp32_over_fp64_batched"] = value / world / comp["fp64_batched"]
        line["comparators"] = comp
        line["dG_err"] = free_energy_error(N)
        line["precision_errors"] = precision_errors(N)
        line["differentiation"] = differentiation_throughput(N, torch)
        line["dcci_batched"] = dcci_batched_throughput(N, torch)
        line["rs_npt_batched"] = rs_npt_batched_throughput(N, torch)
        cps, nst, dt = cpu_baseline_sample()
        line["cpu_baseline"] = {"value": cps, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "host_cores_available": os.cpu_count(),
                                "sample": f"{nst} FP64-oracle MD steps of one 8000-atom replica ({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Seeded synthetic inputs: lattices, liquid-like configurations, velocities, sizes.

This module holds none of the method's arithmetic (no potential, integrator, schedule or
estimator); it only lays out atoms and draws random numbers, so both the CUDA path and
the FP64 oracle may be fed from it.  Positions are (n, 3) float64 arrays in Angstrom,
boxes are orthorhombic (3,) float64 arrays.  Every generator is deterministic in its seed.

Structures follow standard crystallography (not the paper, which only names the phases):
  * diamond (Si-cd): conventional cubic cell, 8 atoms, fcc + (1/4, 1/4, 1/4);
  * beta-tin (A5, I4_1/amd): conventional tetragonal cell, 4 atoms at (0,0,0),
    (0,1/2,1/4), (1/2,1/2,1/2), (1/2,0,3/4);
  * liquid: uniform random positions at a given number density with a minimum pair
    separation enforced by rejection.
"""
from __future__ import annotations

import math

import numpy as np

DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])
BETA_SN_BASIS = np.array([
    [0.0, 0.0, 0.00], [0.0, 0.5, 0.25], [0.5, 0.5, 0.50], [0.5, 0.0, 0.75],
])


def _lattice(basis, cell, nx, ny, nz):
    cell = np.asarray(cell, dtype=np.float64)
    idx = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1)
    idx = idx.reshape(-1, 1, 3).astype(np.float64)
    pos = (idx + basis[None, :, :]) * cell[None, None, :]
    box = cell * np.array([nx, ny, nz], dtype=np.float64)
    return pos.reshape(-1, 3).copy(), box


def diamond(nx: int, ny: int, nz: int, a: float = 5.431):
    """Diamond-cubic crystal of nx*ny*nz conventional cells (8 nx ny nz atoms)."""
    return _lattice(DIAMOND_BASIS, (a, a, a), nx, ny, nz)


def beta_tin(nx: int, ny: int, nz: int, a: float = 4.8, c_over_a: float = 0.55):
    """beta-tin crystal of nx*ny*nz tetragonal cells (4 nx ny nz atoms), c = c_over_a * a."""
    return _lattice(BETA_SN_BASIS, (a, a, a * c_over_a), nx, ny, nz)


def rattle(x, amplitude: float, seed: int):
    """Uniform random displacement in [-amplitude, amplitude]^3 per atom."""
    rng = np.random.Generator(np.random.Philox(seed))
    return x + rng.uniform(-amplitude, amplitude, size=x.shape)


def liquid(n: int, density: float, seed: int, rmin: float = 1.9):
    """n atoms placed uniformly at random in a periodic cube of number density ``density``
    (atoms/A^3), rejecting any trial closer than ``rmin`` (minimum image) to an accepted
    atom.  Returns (positions, box)."""
    L = (n / density) ** (1.0 / 3.0)
    rng = np.random.Generator(np.random.Philox(seed))
    nc = max(1, int(L // rmin))
    h = L / nc
    grid: dict = {}
    pos = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > 200 * n:
            raise RuntimeError("liquid(): rejection sampling did not converge")
        p = rng.uniform(0.0, L, size=3)
        c = tuple((p // h).astype(int) % nc)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    cc = ((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc)
                    for j in grid.get(cc, ()):
                        d = pos[j] - p
                        d -= L * np.rint(d / L)
                        if d @ d < rmin * rmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pos[k] = p
            grid.setdefault(c, []).append(k)
            k += 1
    return pos, np.array([L, L, L])


def gaussian_velocities(n: int, sigma_v: float, seed: int):
    """Velocities with independent N(0, sigma_v^2) components, zero total momentum (equal
    masses), rescaled so that sum |v|^2 = (3n - 3) sigma_v^2 exactly.  With
    sigma_v^2 = kB T / m this is a Maxwell-Boltzmann draw at temperature T exactly."""
    rng = np.random.Generator(np.random.Philox(seed))
    v = rng.standard_normal((n, 3)) * sigma_v
    v -= v.mean(axis=0)
    s2 = float(np.sum(v * v))
    if n > 1 and s2 > 0.0:
        v *= math.sqrt((3 * n - 3) * sigma_v * sigma_v / s2)
    return v


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int):
    """``count`` integers log-uniform in [lo, hi] (the uneven replica sizes of a batch)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))


def diamond_cells_for(n_target: float, min_cells: int = 2):
    """Cell counts (nx, ny, nz) of a diamond crystal with about n_target atoms, as cubic
    as possible, each count >= min_cells."""
    m = max(min_cells ** 3, int(round(n_target / 8.0)))
    nx = max(min_cells, int(round(m ** (1.0 / 3.0))))
    ny = max(min_cells, int(round(math.sqrt(m / nx))))
    nz = max(min_cells, int(round(m / (nx * ny))))
    return nx, ny, nz


def beta_tin_cells_for(n_target: float, c_over_a: float = 0.55, min_xy: int = 2, min_z: int = 4):
    """Cell counts of a beta-tin crystal with about n_target atoms and a near-cubic box."""
    m = max(min_xy * min_xy * min_z, int(round(n_target / 4.0)))
    # box ~ (nx a, ny a, nz c): choose nz ~ nx / c_over_a
    nx = max(min_xy, int(round((m * c_over_a) ** (1.0 / 3.0))))
    nz = max(min_z, int(round(m / (nx * nx))))
    return nx, nx, nz

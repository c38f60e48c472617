"""Gaussian-well model systems that stand in for the paper's materials.

The paper's workloads (molecules, solids, Si nanocrystals, solid/liquid
interfaces; Sec. IV) need pseudopotentials and Quantum ESPRESSO ground
states that are not available here.  They are replaced by local Kohn-Sham
potentials built from randomly placed Gaussian wells, with the grid, cell,
occupied-state count and PDEP count of each workload:

  * ``tiny``      : 24^3 grid, L = 10 bohr cube, 8 wells, N_occ 8, N_pdep 16
  * ``cube48``    : 48^3 grid, L = 20 bohr cube, 64 wells, N_occ 64, N_pdep 128
  * ``uneven``    : 32 systems, N in {24,32,40,48,64}, L = 10 N / 24,
                    N_occ ~ U{8..96}, N_pdep = 2 N_occ, wells ~ volume
  * ``interface`` : 64x64x192 grid, 20x20x60 bohr, a deep dense slab of
                    wells (z < 30) against a shallow sparse one, N_occ 512,
                    N_pdep 512

Each well a contributes  -D_a exp(-|r - R_a - T|^2 / (2 w_a^2))  summed over
lattice translations T.  The image sum is taken per Cartesian axis with a
cut-off |d| < 12 w on each axis; a spherical 12 w cut-off differs from it
only by terms below exp(-72) ~ 5e-32 of the well depth.  Random draws come
from ``numpy.random.default_rng(seed)`` in the order (R, D, w) per well.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1501031410
BATCH_SEED_BASE = 1501031430


@dataclass
class System:
    """One synthetic Kohn-Sham system (input data only)."""

    name: str
    grid: tuple            # (N1, N2, N3); arrays are row-major, N3 fastest
    cell: tuple            # orthorhombic edges (bohr)
    v_r: np.ndarray        # local potential on the grid (Ha), float64, shape grid
    n_occ: int
    n_pdep: int
    seed: int
    wells: list = field(default_factory=list)   # (R, D, w) per well
    cg_tol: float = 1e-10
    n_dav: int = 0          # 0: iterate Davidson to convergence

    @property
    def n_r(self) -> int:
        return int(np.prod(self.grid))


def periodic_gaussian_sum(grid, cell, centres, depths, widths, sign=-1.0):
    """sign * sum_a D_a * exp(-|r - R_a - T|^2 / (2 w_a^2)) on the grid.

    The lattice-image sum is separable per axis: for each axis the 1D
    factor sums exp(-(x - X - m L)^2 / (2 w^2)) over integers m with
    |x - X - m L| < 12 w.
    """
    grid = tuple(int(n) for n in grid)
    cell = tuple(float(l) for l in cell)
    out = np.zeros(grid, dtype=np.float64)
    axes = [np.arange(n, dtype=np.float64) * (l / n) for n, l in zip(grid, cell)]
    for R, D, w in zip(centres, depths, widths):
        factors = []
        for ax in range(3):
            x = axes[ax]
            L = cell[ax]
            cut = 12.0 * w
            mmax = int(np.ceil((cut + L) / L)) + 1
            f = np.zeros_like(x)
            for m in range(-mmax, mmax + 1):
                d = x - R[ax] - m * L
                mask = np.abs(d) < cut
                f[mask] += np.exp(-(d[mask] ** 2) / (2.0 * w * w))
            factors.append(f)
        out += sign * D * (factors[0][:, None, None] * factors[1][None, :, None]
                           * factors[2][None, None, :])
    return out


def gaussian_wells(rng, n_wells, cell, depth, width, zrange=None):
    """Draw n_wells wells in the order (R, D, w) per well.

    zrange, if given, confines the third coordinate of R to [z0, z1).
    """
    centres, depths, widths = [], [], []
    for _ in range(n_wells):
        R = rng.uniform(0.0, 1.0, size=3) * np.asarray(cell, dtype=np.float64)
        if zrange is not None:
            R[2] = zrange[0] + (R[2] / cell[2]) * (zrange[1] - zrange[0])
        D = rng.uniform(depth[0], depth[1])
        w = rng.uniform(width[0], width[1])
        centres.append(R)
        depths.append(D)
        widths.append(w)
    return centres, depths, widths


def _cube_system(name, N, L, n_wells, n_occ, n_pdep, seed, depth=(1.0, 3.0),
                 width=(0.8, 1.5), n_dav=0, cg_tol=1e-10):
    rng = np.random.default_rng(seed)
    cell = (L, L, L)
    c, d, w = gaussian_wells(rng, n_wells, cell, depth, width)
    v = periodic_gaussian_sum((N, N, N), cell, c, d, w)
    return System(name=name, grid=(N, N, N), cell=cell, v_r=v, n_occ=n_occ,
                  n_pdep=n_pdep, seed=seed, wells=list(zip(c, d, w)),
                  cg_tol=cg_tol, n_dav=n_dav)


def _interface_system(seed):
    rng = np.random.default_rng(seed)
    cell = (20.0, 20.0, 60.0)
    grid = (64, 64, 192)
    # base density of the 48^3 workload: 64 wells per 8000 bohr^3; each half
    # cell is 12000 bohr^3 -> 96 wells, doubled (deep side) or halved.
    c1, d1, w1 = gaussian_wells(rng, 192, cell, (2.0, 4.0), (0.8, 1.5), zrange=(0.0, 30.0))
    c2, d2, w2 = gaussian_wells(rng, 48, cell, (0.5, 1.5), (0.8, 1.5), zrange=(30.0, 60.0))
    c, d, w = c1 + c2, d1 + d2, w1 + w2
    v = periodic_gaussian_sum(grid, cell, c, d, w)
    return System(name="interface", grid=grid, cell=cell, v_r=v, n_occ=512,
                  n_pdep=512, seed=seed, wells=list(zip(c, d, w)), n_dav=6)


#: workload name -> (description, builder)
WORKLOADS = {
    "tiny": "24^3 grid, L=10 bohr, 8 wells, N_occ=8, N_pdep=16, Davidson to convergence",
    "cube48": "48^3 grid, L=20 bohr, 64 wells, N_occ=64, N_pdep=128, 6 Davidson iterations",
    "uneven": "32 systems, N in {24,32,40,48,64}, L=10N/24, N_occ~U{8..96}, N_pdep=2N_occ",
    "interface": "64x64x192 grid, 20x20x60 bohr, two slabs of wells, N_occ=512, N_pdep=512",
}


def make_system(name: str, seed: int | None = None) -> System:
    """Build one named workload deterministically from its seed."""
    if name == "tiny":
        return _cube_system("tiny", 24, 10.0, 8, 8, 16,
                            SEED_BASE + 0 if seed is None else seed)
    if name == "cube48":
        return _cube_system("cube48", 48, 20.0, 64, 64, 128,
                            SEED_BASE + 1 if seed is None else seed, n_dav=6)
    if name == "interface":
        return _interface_system(SEED_BASE + 4 if seed is None else seed)
    raise ValueError(f"unknown workload {name!r}")


def make_batch(n_systems: int = 32, seed0: int = BATCH_SEED_BASE, grids=(24, 32, 40, 48, 64)):
    """The uneven batch: system k is drawn from seed0 + k."""
    out = []
    for k in range(n_systems):
        rng = np.random.default_rng(seed0 + k)
        N = int(rng.choice(np.asarray(grids)))
        n_occ = int(rng.integers(8, 97))
        L = N * 10.0 / 24.0
        n_wells = int(round(8.0 * (L / 10.0) ** 3))
        cell = (L, L, L)
        c, d, w = gaussian_wells(rng, n_wells, cell, (1.0, 3.0), (0.8, 1.5))
        v = periodic_gaussian_sum((N, N, N), cell, c, d, w)
        out.append(System(name=f"uneven{k}", grid=(N, N, N), cell=cell, v_r=v,
                          n_occ=n_occ, n_pdep=2 * n_occ, seed=seed0 + k,
                          wells=list(zip(c, d, w)), n_dav=6))
    return out


def random_vectors(seed: int, n: int, dim: int) -> np.ndarray:
    """n standard-normal vectors of length dim, shape (n, dim), float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, dim))


def random_grid_potentials(seed: int, n: int, grid, cell, n_bumps: int = 4) -> np.ndarray:
    """n smooth random perturbing potentials dV(r) (Ha), shape (n, *grid).

    Each is a sum of n_bumps periodic Gaussians with centres ~ U(cell),
    signed amplitudes ~ U[-1, 1] Ha and widths ~ U[1, 2] bohr.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((n,) + tuple(grid), dtype=np.float64)
    for j in range(n):
        c, d, w = gaussian_wells(rng, n_bumps, cell, (-1.0, 1.0), (1.0, 2.0))
        out[j] = periodic_gaussian_sum(grid, cell, c, d, w, sign=1.0)
    return out

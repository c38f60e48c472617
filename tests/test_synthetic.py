"""The seeded input generators (synthetic/): the recipe of each workload and
the periodic Gaussian-well sum against a brute-force lattice sum."""
import itertools

import numpy as np
import pytest

import synthetic


def _brute_force_wells(grid, cell, centres, depths, widths):
    """-sum_a D_a exp(-|r - R_a - T|^2 / (2 w_a^2)) over lattice vectors T
    with a spherical cut-off |r - R_a - T| < 12 w_a, point by point."""
    axes = [np.arange(n) * (l / n) for n, l in zip(grid, cell)]
    r = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    out = np.zeros(grid)
    L = np.asarray(cell)
    for R, D, w in zip(centres, depths, widths):
        m = [int(np.ceil(12 * w / l)) + 1 for l in cell]
        for t in itertools.product(*[range(-k, k + 1) for k in m]):
            d = r - np.asarray(R) - np.asarray(t) * L
            d2 = np.sum(d * d, axis=-1)
            out -= np.where(d2 < (12 * w) ** 2, D * np.exp(-d2 / (2 * w * w)), 0.0)
    return out


def test_periodic_sum_against_brute_force():
    grid, cell = (12, 10, 14), (6.0, 5.0, 7.0)
    rng = np.random.default_rng(3)
    c, d, w = synthetic.gaussian_wells(rng, 3, cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(grid, cell, c, d, w)
    ref = _brute_force_wells(grid, cell, c, d, w)
    assert np.abs(v - ref).max() < 1e-13 * np.abs(ref).max()
    # periodic: a well moved by a lattice vector gives the same potential
    c2 = [np.asarray(R) + np.array([cell[0], -2 * cell[1], cell[2]]) for R in c]
    assert np.abs(synthetic.periodic_gaussian_sum(grid, cell, c2, d, w) - v).max() < 1e-12


def test_draw_order_and_ranges():
    rng = np.random.default_rng(11)
    c, d, w = synthetic.gaussian_wells(rng, 5, (10.0, 10.0, 10.0), (1.0, 3.0), (0.8, 1.5))
    rng = np.random.default_rng(11)
    for R, D, W in zip(c, d, w):
        np.testing.assert_array_equal(R, rng.uniform(0.0, 1.0, size=3) * 10.0)
        assert D == rng.uniform(1.0, 3.0) and W == rng.uniform(0.8, 1.5)


@pytest.mark.parametrize("name,grid,L,wells,n_occ,n_pdep", [
    ("tiny", (24, 24, 24), 10.0, 8, 8, 16),
    ("cube48", (48, 48, 48), 20.0, 64, 64, 128),
])
def test_cube_workloads(name, grid, L, wells, n_occ, n_pdep):
    s = synthetic.make_system(name)
    assert s.grid == grid and s.cell == (L, L, L)
    assert (s.n_occ, s.n_pdep) == (n_occ, n_pdep) and len(s.wells) == wells
    assert s.v_r.shape == grid and s.v_r.dtype == np.float64 and s.v_r.max() <= 0.0
    for R, D, w in s.wells:
        assert np.all((0 <= R) & (R < L)) and 1.0 <= D <= 3.0 and 0.8 <= w <= 1.5
    again = synthetic.make_system(name)
    np.testing.assert_array_equal(again.v_r, s.v_r)
    assert not np.array_equal(synthetic.make_system(name, seed=s.seed + 1).v_r, s.v_r)


def test_uneven_batch_recipe():
    batch = synthetic.make_batch(8)
    for k, s in enumerate(batch):
        N = s.grid[0]
        L = N * 10.0 / 24.0
        assert s.grid == (N, N, N) and N in (24, 32, 40, 48, 64)
        assert s.cell == pytest.approx((L, L, L))
        assert 8 <= s.n_occ <= 96 and s.n_pdep == 2 * s.n_occ
        assert len(s.wells) == int(round(8.0 * (L / 10.0) ** 3))
        assert s.seed == synthetic.systems.BATCH_SEED_BASE + k


def test_interface_recipe():
    s = synthetic.make_system("interface")
    assert s.grid == (64, 64, 192) and s.cell == (20.0, 20.0, 60.0)
    assert (s.n_occ, s.n_pdep) == (512, 512)
    deep = [(R, D) for R, D, _ in s.wells if R[2] < 30.0]
    shallow = [(R, D) for R, D, _ in s.wells if R[2] >= 30.0]
    assert len(deep) == 192 and len(shallow) == 48
    assert all(2.0 <= D <= 4.0 for _, D in deep) and all(0.5 <= D <= 1.5 for _, D in shallow)
    # the deep slab is deeper on average
    z = np.arange(192) * (60.0 / 192)
    prof = s.v_r.mean(axis=(0, 1))
    assert prof[z < 30].mean() < 2 * prof[z >= 30].mean()


def test_random_inputs_are_seeded():
    a = synthetic.random_vectors(4, 3, 50)
    np.testing.assert_array_equal(a, synthetic.random_vectors(4, 3, 50))
    assert a.shape == (3, 50)
    p = synthetic.random_grid_potentials(6, 2, (12, 12, 12), (6.0, 6.0, 6.0))
    assert p.shape == (2, 12, 12, 12)
    np.testing.assert_array_equal(p, synthetic.random_grid_potentials(6, 2, (12, 12, 12),
                                                                      (6.0, 6.0, 6.0)))

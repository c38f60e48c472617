"""Pins of the oracle's plane-wave sphere and real-coefficient layout.

The sphere counts are fixed by the grid rule r_i = (N_i - 1)/4 and the
cells of the workloads; the real layout is checked against cos/sin basis
functions evaluated directly on the grid (no FFT involved).
"""
import numpy as np
import pytest

from oracle.basis import Basis, derived_ecut


def _brute_count(grid, cell):
    ecut = derived_ecut(grid, cell)
    cnt = 0
    rng = [range(-(n // 2) + 1, n // 2) for n in grid]
    for a in rng[0]:
        for b in rng[1]:
            for c in rng[2]:
                g2 = sum((2 * np.pi * k / L) ** 2 for k, L in zip((a, b, c), cell))
                if 0.5 * g2 <= ecut:
                    cnt += 1
    return cnt


@pytest.mark.parametrize("grid,cell,npw", [
    ((24, 24, 24), (10.0, 10.0, 10.0), 799),
    ((48, 48, 48), (20.0, 20.0, 20.0), 6859),
    ((64, 64, 192), (20.0, 20.0, 60.0), 49095),
])
def test_sphere_sizes(grid, cell, npw):
    b = Basis(grid, cell)
    assert b.n_pw == npw
    assert b.n_pw == 2 * b.n_half + 1
    if np.prod(grid) <= 24 ** 3:
        assert _brute_count(grid, cell) == npw


def test_half_space_order():
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    h = b.half
    # strictly increasing in (n3, n2, n1)
    keys = [(n[2], n[1], n[0]) for n in h]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # half space: no member's mirror is a member, and mirrors cover the rest
    s = set(map(tuple, h))
    assert all(tuple(-np.asarray(n)) not in s for n in h)
    assert (0, 0, 0) not in s


def test_real_layout_is_cos_sin():
    """x = e_{2k} is sqrt2 cos(G_k.r); x = e_{2k+1} is -sqrt2 sin(G_k.r)."""
    b = Basis((12, 12, 12), (6.0, 7.0, 8.0))
    N = np.asarray(b.grid)
    L = np.asarray(b.cell)
    idx = np.indices(b.grid).reshape(3, -1).T
    r = idx * (L / N)[None, :]
    for k in [0, 3, b.n_half - 1]:
        G = 2 * np.pi * b.half[k] / L
        ph = r @ G
        x = np.zeros(b.n_pw)
        x[2 * k] = 1.0
        u = b.coeffs_to_grid(x).ravel()
        np.testing.assert_allclose(u, np.sqrt(2) * np.cos(ph), atol=1e-13)
        x[:] = 0.0
        x[2 * k + 1] = 1.0
        u = b.coeffs_to_grid(x).ravel()
        np.testing.assert_allclose(u, -np.sqrt(2) * np.sin(ph), atol=1e-13)
    x = np.zeros(b.n_pw)
    x[-1] = 1.0
    np.testing.assert_allclose(b.coeffs_to_grid(x).ravel(), 1.0, atol=1e-14)


def test_roundtrip_and_inner_product():
    b = Basis((16, 16, 16), (7.0, 7.0, 7.0))
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, b.n_pw))
    u = b.coeffs_to_grid(x)
    np.testing.assert_allclose(b.grid_to_coeffs(u), x, atol=1e-12)
    # Euclidean dot of coefficients = L2 inner product of Omega^{-1/2} u
    ip = np.sum(u[0] * u[1]) / b.n_r
    assert abs(ip - x[0] @ x[1]) < 1e-11 * np.linalg.norm(x[0]) * np.linalg.norm(x[1])

"""Pins of the oracle's dense Hamiltonian (Sec. II, local potential).

* matrix elements against explicit grid quadrature of cos/sin basis
  functions (catches a wrong sign or index in V(G - G'));
* V = 0: eigenvalues are the sorted kinetic energies 1/2|G|^2;
* V -> V + c shifts every eigenvalue by c and leaves the states unchanged;
* H applied through grid products equals the dense matrix.
"""
import numpy as np

import synthetic
from oracle.basis import Basis
from oracle.hamiltonian import apply_hamiltonian_grid, dense_hamiltonian, ks_states


def _real_basis_functions(b):
    """u_p(r) for every real component p, from explicit cos/sin formulas."""
    N = np.asarray(b.grid)
    L = np.asarray(b.cell)
    r = np.indices(b.grid).reshape(3, -1).T * (L / N)[None, :]
    out = np.empty((b.n_pw, b.n_r))
    for k, n in enumerate(b.half):
        ph = r @ (2 * np.pi * n / L)
        out[2 * k] = np.sqrt(2) * np.cos(ph)
        out[2 * k + 1] = -np.sqrt(2) * np.sin(ph)
    out[-1] = 1.0
    return out


def test_matrix_elements_brute_force():
    grid, cell = (9, 9, 9), (5.0, 5.5, 6.0)
    b = Basis(grid, cell)
    rng = np.random.default_rng(11)
    c, d, w = synthetic.gaussian_wells(rng, 3, cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(grid, cell, c, d, w)
    u = _real_basis_functions(b)
    # <b_p|V|b_q> = (Omega/N_r) sum_k Omega^{-1} u_p V u_q
    ref = (u * v.ravel()[None, :]) @ u.T / b.n_r
    ref[np.diag_indices_from(ref)] += 0.5 * b.g2_real
    h = dense_hamiltonian(b, v)
    np.testing.assert_allclose(h, ref, atol=1e-12)


def test_free_electron_spectrum():
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    ks = ks_states(b, np.zeros(b.grid), 7)
    np.testing.assert_allclose(ks.eps, np.sort(0.5 * b.g2_full), atol=1e-12)


def test_constant_shift(tiny_system):
    b = Basis((16, 16, 16), (7.0, 7.0, 7.0))
    rng = np.random.default_rng(5)
    c, d, w = synthetic.gaussian_wells(rng, 4, b.cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(b.grid, b.cell, c, d, w)
    k1 = ks_states(b, v, 4)
    k2 = ks_states(b, v + 0.37, 4)
    np.testing.assert_allclose(k2.eps, k1.eps + 0.37, atol=1e-11)
    ov = np.abs(np.sum(k1.C[:, :4] * k2.C[:, :4], axis=0))
    np.testing.assert_allclose(ov, 1.0, atol=1e-9)


def test_grid_application_matches_dense(tiny_oracle, tiny_system):
    b, _, h = tiny_oracle
    x = np.random.default_rng(2).standard_normal((3, b.n_pw))
    hx = apply_hamiltonian_grid(b, tiny_system.v_r, x)
    np.testing.assert_allclose(hx, x @ h, atol=1e-12 * np.abs(hx).max())


def test_tiny_has_a_gap(tiny_oracle):
    _, ks, _ = tiny_oracle
    assert ks.gap > 1e-3

"""Pins of the oracle's large-system routes (oracle/iterative.py).

Each route is checked against the dense route it replaces, on systems where
both run: the real-FFT grid transforms against the complex-FFT ones of
oracle.basis (cubic and non-cubic grids, which exercise the n3 = 0 mirror
plane), the block H application against apply_hamiltonian_grid and the
dense matrix, the Lanczos eigenpairs against dense eigh, the preconditioned
block CG solutions of Eq. stern against the sum over all empty states, and
chi0bar phi and dn(r) against response.chi0bar_apply.  Planted mistakes (a
dropped n3 = 0 mirror, a wrong occupied energy) are caught.
"""
import numpy as np
import pytest

import synthetic
from oracle import iterative as it
from oracle.basis import Basis
from oracle.hamiltonian import apply_hamiltonian_grid, dense_hamiltonian, ks_states
from oracle.response import chi0bar_apply, sternheimer_sos


@pytest.fixture(scope="module")
def tiny():
    s = synthetic.make_system("tiny")
    b = Basis(s.grid, s.cell)
    return s, b, ks_states(b, s.v_r, s.n_occ)


@pytest.mark.parametrize("grid,cell", [((24, 24, 24), (10.0, 10.0, 10.0)),
                                       ((16, 20, 32), (7.0, 9.0, 13.0))])
def test_transforms_match_complex_fft(grid, cell):
    b = Basis(grid, cell)
    x = np.random.default_rng(7).standard_normal((5, b.n_pw))
    u = it.to_grid(b, x)
    assert np.abs(u - b.coeffs_to_grid(x)).max() < 1e-12 * np.abs(u).max()
    assert np.abs(it.from_grid(b, u) - x).max() < 1e-12
    assert np.abs(it.from_grid(b, u) - b.grid_to_coeffs(u)).max() < 1e-12


def test_missing_mirror_plane_is_caught():
    b = Basis((16, 20, 32), (7.0, 9.0, 13.0))
    x = np.random.default_rng(8).standard_normal((2, b.n_pw))
    ref = b.coeffs_to_grid(x)
    orig = it._half_index

    def broken(basis):
        pos, m0, mpos = orig(basis)
        return pos, m0[:0], tuple(a[:0] for a in mpos)

    it._half_index = broken
    try:
        bad = it.to_grid(b, x)
    finally:
        it._half_index = orig
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


def test_block_hamiltonian(tiny):
    s, b, _ = tiny
    x = np.random.default_rng(9).standard_normal((4, b.n_pw))
    hx = it.apply_h(b, s.v_r, x)
    assert np.abs(hx - apply_hamiltonian_grid(b, s.v_r, x)).max() < 1e-12 * np.abs(hx).max()
    h = dense_hamiltonian(b, s.v_r)
    assert np.abs(hx - x @ h).max() < 1e-11 * np.abs(hx).max()


def test_lanczos_states_match_dense_eigh(tiny):
    s, b, ks = tiny
    kl = it.ks_states_lanczos(b, s.v_r, s.n_occ, n_states=s.n_occ + 4)
    assert np.abs(kl.eps - ks.eps[: s.n_occ + 4]).max() < 1e-11
    # the occupied subspace (projector) is the same
    Pa = kl.C[:, : s.n_occ] @ kl.C[:, : s.n_occ].T
    Pb = ks.C[:, : s.n_occ] @ ks.C[:, : s.n_occ].T
    assert np.abs(Pa - Pb).max() < 1e-10
    res = it.apply_h(b, s.v_r, kl.C.T) - kl.eps[:, None] * kl.C.T
    assert np.linalg.norm(res, axis=1).max() < 1e-10


def test_pcg_equals_sum_over_states(tiny):
    s, b, ks = tiny
    dv = synthetic.random_grid_potentials(5, 1, s.grid, s.cell)[0]
    x, its, res = it.sternheimer_pcg(b, ks, s.v_r, dv, tol=1e-12)
    ref = sternheimer_sos(b, ks, dv)
    assert res.max() < 1e-11 and its.min() > 0
    assert np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    # a subset of states leaves the other rows zero and the listed ones equal
    xs, _, _ = it.sternheimer_pcg(b, ks, s.v_r, dv, states=[0, 5], tol=1e-12)
    assert np.abs(xs[[0, 5]] - ref[[0, 5]]).max() < 1e-10 * np.abs(ref).max()
    assert not xs[[1, 2, 3, 4, 6, 7]].any()


def test_pcg_wrong_state_energy_is_caught(tiny):
    s, b, ks = tiny
    dv = synthetic.random_grid_potentials(6, 1, s.grid, s.cell)[0]
    ref = sternheimer_sos(b, ks, dv)
    # eps_v off by 10 mHa (e.g. a unit or index slip) must not reproduce Eq. stern
    bad = type(ks)(eps=ks.eps + 0.01, C=ks.C, n_occ=ks.n_occ)
    x, _, _ = it.sternheimer_pcg(b, bad, s.v_r, dv, tol=1e-12)
    assert np.abs(x - ref).max() > 1e-3 * np.abs(ref).max()


def test_chi0bar_pcg_equals_sum_over_states(tiny):
    s, b, ks = tiny
    phi = synthetic.random_vectors(3, 2, b.n_pdep_dim)
    c1, n1 = it.chi0bar_apply_pcg(b, ks, s.v_r, phi, tol=1e-12, return_dn=True)
    c0, n0 = chi0bar_apply(b, ks, phi, return_dn=True)
    assert np.abs(c1 - c0).max() < 1e-10 * np.abs(c0).max()
    assert np.abs(n1 - n0).max() < 1e-10 * np.abs(n0).max()
    # with Lanczos states (only the occupied block and one empty state known)
    kl = it.ks_states_lanczos(b, s.v_r, s.n_occ)
    c2 = it.chi0bar_apply_pcg(b, kl, s.v_r, phi, tol=1e-12)
    assert np.abs(c2 - c0).max() < 1e-10 * np.abs(c0).max()

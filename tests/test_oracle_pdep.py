"""Pins of the oracle's dense chi0bar and PDEP reference (Secs. II A to II C).

* V = 0 closed form, diagonal in G, for closed shells (factors 4, 4 pi,
  Omega, sign and the sqrt(4 pi)/|G| symmetrisation all enter);
* chi0bar is symmetric and negative semi-definite (Eq. AdlerWiser at
  omega = 0: every term is -|p|^2 / (eps_c - eps_v));
* chi0bar applied through Sternheimer solves equals the dense matrix;
* invariance under V -> V + const and under rotations inside degenerate
  shells;
* planted mistakes in the oracle (a wrong Coulomb root, a dropped factor)
  are caught by these pins.
"""
import numpy as np
import pytest

import synthetic
from oracle import response
from oracle.basis import Basis
from oracle.hamiltonian import ks_states
from oracle.pdep import chi0bar_dense, free_electron_chi0bar, pdep_reference


@pytest.mark.parametrize("n_occ", [1, 7, 19])
def test_free_electron_closed_form(n_occ):
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    ks = ks_states(b, np.zeros(b.grid), n_occ)
    chib = chi0bar_dense(b, ks)
    lam = free_electron_chi0bar(b, n_occ)
    scale = np.abs(lam).max()
    np.testing.assert_allclose(chib, np.diag(lam), atol=1e-13 * scale)


def test_free_electron_anisotropic_cell():
    b = Basis((12, 12, 16), (6.0, 6.0, 8.5))
    g2 = np.sort(0.5 * b.g2_full)
    # first closed shell above the ground state
    n_occ = int(np.searchsorted(g2, g2[1] + 1e-9))
    ks = ks_states(b, np.zeros(b.grid), n_occ)
    chib = chi0bar_dense(b, ks)
    lam = free_electron_chi0bar(b, n_occ)
    np.testing.assert_allclose(chib, np.diag(lam), atol=1e-13 * np.abs(lam).max())


def test_symmetric_nsd(tiny_chib):
    chib = tiny_chib
    assert np.abs(chib - chib.T).max() < 1e-14 * np.abs(chib).max()
    lam = np.linalg.eigvalsh(0.5 * (chib + chib.T))
    assert lam.max() <= 1e-12 * abs(lam.min())
    assert lam.min() < 0


def test_sternheimer_route_equals_dense(tiny_oracle, tiny_chib):
    b, ks, _ = tiny_oracle
    phi = synthetic.random_vectors(9, 3, b.n_pdep_dim)
    out = response.chi0bar_apply(b, ks, phi)
    np.testing.assert_allclose(out, phi @ tiny_chib, atol=1e-12 * np.abs(out).max())


def test_constant_shift_invariance():
    b = Basis((16, 16, 16), (7.0, 7.0, 7.0))
    rng = np.random.default_rng(8)
    c, d, w = synthetic.gaussian_wells(rng, 4, b.cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(b.grid, b.cell, c, d, w)
    l1, _ = pdep_reference(chi0bar_dense(b, ks_states(b, v, 4)), 8)
    l2, _ = pdep_reference(chi0bar_dense(b, ks_states(b, v - 1.3, 4)), 8)
    np.testing.assert_allclose(l2, l1, rtol=1e-11)


def test_degenerate_shell_rotation_invariance():
    """chi0bar depends on the occupied and empty spaces, not on the basis chosen
    inside a degenerate shell: random rotations of the six degenerate
    |k| = 2 pi/L free-electron states (occupied) and of the twelve of the next
    shell (empty) leave it unchanged, while the same rotation mixing occupied
    and empty states does not."""
    from oracle.hamiltonian import KSStates
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    ks = ks_states(b, np.zeros(b.grid), 7)
    assert np.ptp(ks.eps[1:7]) < 1e-12 and np.ptp(ks.eps[7:19]) < 1e-12
    ref = chi0bar_dense(b, ks)
    rng = np.random.default_rng(5)
    C = ks.C.copy()
    for lo, hi in ((1, 7), (7, 19)):
        q, _ = np.linalg.qr(rng.standard_normal((hi - lo, hi - lo)))
        C[:, lo:hi] = C[:, lo:hi] @ q
    rot = chi0bar_dense(b, KSStates(eps=ks.eps, C=C, n_occ=7))
    scale = np.abs(ref).max()
    assert np.abs(rot - ref).max() < 1e-13 * scale
    # mixing an occupied state with an empty one changes the response
    C2 = ks.C.copy()
    c, s_ = np.cos(0.3), np.sin(0.3)
    C2[:, [6, 7]] = C2[:, [6, 7]] @ np.array([[c, -s_], [s_, c]])
    mixed = chi0bar_dense(b, KSStates(eps=ks.eps, C=C2, n_occ=7))
    assert np.abs(mixed - ref).max() > 1e-3 * scale


def test_tiny_reference_shape(tiny_chib, tiny_system):
    lam, vec = pdep_reference(tiny_chib, tiny_system.n_pdep)
    assert lam.shape == (16,) and vec.shape == (798, 16)
    assert np.all(np.diff(lam) >= 0)
    assert lam[-1] < 0


def test_planted_coulomb_root_is_caught(monkeypatch):
    """A wrong v^{1/2} (4 pi/|G| instead of sqrt(4 pi)/|G|) fails the closed form."""
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    ks = ks_states(b, np.zeros(b.grid), 7)
    lam = free_electron_chi0bar(b, 7)
    monkeypatch.setattr(Basis, "sqrt_coulomb",
                        lambda self: 4.0 * np.pi / np.sqrt(self.g2_real[:-1]))
    chib = chi0bar_dense(b, ks)
    assert np.abs(chib - np.diag(lam)).max() > 1e-3 * np.abs(lam).max()


def test_planted_spin_factor_is_caught(monkeypatch, tiny_oracle, tiny_system):
    """Dropping the spin factor in dn fails the finite-difference density pin."""
    b, ks, _ = tiny_oracle
    dv = synthetic.random_grid_potentials(79, 1, tiny_system.grid, tiny_system.cell)[0]
    orig = response.density_response
    monkeypatch.setattr(response, "density_response",
                        lambda basis, u, dpsi: 0.5 * orig(basis, u, dpsi))
    eta = 1e-4
    n_p = response.density_from_states(b, ks_states(b, tiny_system.v_r + eta * dv, ks.n_occ))
    n_m = response.density_from_states(b, ks_states(b, tiny_system.v_r - eta * dv, ks.n_occ))
    fd = (n_p - n_m) / (2 * eta)
    dn = response.density_response(b, response.occupied_grid(b, ks),
                                   response.sternheimer_sos(b, ks, dv))
    assert np.linalg.norm(fd - dn) / np.linalg.norm(fd) > 0.1

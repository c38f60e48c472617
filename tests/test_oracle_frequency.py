"""Pins of the oracle's chi0bar at imaginary frequency and of B, Lambda (Sec. II B).

* V = 0 closed form at omega = i nu (1e-13): the diagonal free-electron
  eigenvalues with (eps_k - eps_{k+G}) / ((eps_k - eps_{k+G})^2 + nu^2);
* continuity at nu -> 0 with the static chi0bar;
* symmetric, negative semidefinite, and monotone in nu as an operator
  (chi0bar(i nu2) - chi0bar(i nu1) is NSD for nu2 < nu1);
* B(0) in the PDEP basis is diag(lambda); Lambda = (1 - B)^{-1} B has the
  eigenvalues b/(1 - b) of B and shares its eigenvectors;
* the free-electron Lambda(i nu) is diag(lambda/(1 - lambda)) of the closed form;
* a planted sign mistake in the imaginary-frequency denominator is caught.
"""
import numpy as np
import pytest

from oracle import screening
from oracle.basis import Basis
from oracle.hamiltonian import ks_states
from oracle.pdep import chi0bar_dense, free_electron_chi0bar, pdep_reference


@pytest.fixture(scope="module")
def free19():
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    return b, ks_states(b, np.zeros(b.grid), 19)


@pytest.mark.parametrize("nu", [0.3, 1.0, 4.0])
def test_free_electron_imaginary_frequency(nu, free19):
    b, ks = free19
    chib = chi0bar_dense(b, ks, nu=nu)
    lam = free_electron_chi0bar(b, 19, nu=nu)
    np.testing.assert_allclose(chib, np.diag(lam), atol=1e-13 * np.abs(lam).max())
    lb = screening.lambda_body(chib)
    np.testing.assert_allclose(lb, np.diag(lam / (1 - lam)), atol=1e-12)


def test_continuity_at_zero(tiny_oracle, tiny_chib):
    b, ks, _ = tiny_oracle
    c = chi0bar_dense(b, ks, nu=1e-7)
    assert np.abs(c - tiny_chib).max() < 1e-9 * np.abs(tiny_chib).max()


def test_symmetric_nsd_monotone(tiny_oracle):
    b, ks, _ = tiny_oracle
    c1 = chi0bar_dense(b, ks, nu=1.0)
    c2 = chi0bar_dense(b, ks, nu=0.25)
    scale = np.abs(c2).max()
    assert np.abs(c1 - c1.T).max() < 1e-14 * scale
    assert np.linalg.eigvalsh(c1).max() <= 1e-12 * scale
    assert np.linalg.eigvalsh(0.5 * ((c2 - c1) + (c2 - c1).T)).max() <= 1e-12 * scale
    assert np.abs(c1).max() < np.abs(c2).max()


def test_body_at_zero_and_lambda(tiny_oracle, tiny_chib, tiny_system):
    b, ks, _ = tiny_oracle
    lam, vec = pdep_reference(tiny_chib, tiny_system.n_pdep)
    B0 = screening.pdep_body(tiny_chib, vec)
    np.testing.assert_allclose(B0, np.diag(lam), atol=1e-12 * np.abs(lam).max())
    B = screening.pdep_body(chi0bar_dense(b, ks, nu=0.5), vec)
    L = screening.lambda_body(B)
    mu, V = np.linalg.eigh(0.5 * (B + B.T))
    np.testing.assert_allclose(V.T @ L @ V, np.diag(mu / (1 - mu)), atol=1e-12)


def test_planted_denominator_sign_is_caught(monkeypatch, free19):
    """den/(den^2 - nu^2) in place of den/(den^2 + nu^2) fails the closed form."""
    from oracle import pdep
    b, ks = free19
    nu = 1.0
    lam = free_electron_chi0bar(b, 19, nu=nu)
    monkeypatch.setattr(pdep, "resolvent_weight", lambda den, nu: den / (den * den - nu * nu))
    chib = pdep.chi0bar_dense(b, ks, nu=nu)
    assert np.abs(chib - np.diag(lam)).max() > 1e-2 * np.abs(lam).max()

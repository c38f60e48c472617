"""Pins of the oracle's reducible chibar, epsbar^{-1} and W^p at omega = 0 (Sec. II A).

* V = 0 closed form: chi0bar is diagonal with the free-electron lambda(G),
  so the Dyson solve must give lambda/(1 - lambda) on the diagonal and W^p
  must equal (4 pi/|G|^2) lambda/(1 - lambda) with |G| taken from the
  integer G vectors (not from the oracle's Coulomb helper);
* the unsymmetrised Dyson equation chi = chi0 + chi0 v chi holds for the
  oracle's chibar mapped back with v^{-1/2};
* epsbar^{-1} (1 - chi0bar) = 1 (the RPA epsbar = 1 - chi0bar);
* chibar and chi0bar share eigenvectors, with eigenvalues lambda/(1-lambda);
* the full-rank PDEP form equals the dense definition for all three kinds;
* spectra: chibar in (-1, 0], epsbar^{-1} in (0, 1] (chi0bar is NSD);
* a planted sign mistake in the Dyson solve is caught.
"""
import numpy as np
import pytest

from oracle import screening
from oracle.basis import Basis
from oracle.hamiltonian import ks_states
from oracle.pdep import chi0bar_dense, free_electron_chi0bar, pdep_reference


@pytest.fixture(scope="module")
def free7():
    b = Basis((12, 12, 12), (6.0, 6.0, 6.0))
    ks = ks_states(b, np.zeros(b.grid), 7)
    return b, chi0bar_dense(b, ks), free_electron_chi0bar(b, 7)


def test_free_electron_dyson(free7):
    b, chib, lam = free7
    chi = screening.chibar_dyson(chib)
    np.testing.assert_allclose(chi, np.diag(lam / (1.0 - lam)), atol=1e-13)
    np.testing.assert_allclose(screening.epsinv_dense(chib), np.diag(1.0 / (1.0 - lam)),
                               atol=1e-13)


def test_free_electron_wp(free7):
    b, chib, lam = free7
    L = np.asarray(b.cell)
    g2 = np.repeat(np.sum((2 * np.pi * b.half / L) ** 2, axis=1), 2)
    wp = screening.wp_dense(b, chib)
    expect = 4.0 * np.pi / g2 * lam / (1.0 - lam)
    np.testing.assert_allclose(wp, np.diag(expect), atol=1e-12 * np.abs(expect).max())


def test_unsymmetrised_dyson(tiny_oracle, tiny_chib):
    b, _, _ = tiny_oracle
    d = b.sqrt_coulomb()
    chi0 = tiny_chib / d[:, None] / d[None, :]
    chi = screening.chibar_dyson(tiny_chib) / d[:, None] / d[None, :]
    v = d * d
    res = chi - chi0 - chi0 @ (v[:, None] * chi)
    assert np.abs(res).max() <= 1e-11 * np.abs(chi).max()


def test_epsinv_inverts_eps(tiny_chib):
    n = tiny_chib.shape[0]
    prod = screening.epsinv_dense(tiny_chib) @ (np.eye(n) - tiny_chib)
    assert np.abs(prod - np.eye(n)).max() < 1e-12


def test_shared_eigenvectors_and_spectra(tiny_chib):
    lam, vec = pdep_reference(tiny_chib, tiny_chib.shape[0])
    chi = screening.chibar_dyson(tiny_chib)
    np.testing.assert_allclose(chi @ vec[:, :40], vec[:, :40] * (lam[:40] / (1 - lam[:40])),
                               atol=1e-12)
    mu = np.linalg.eigvalsh(0.5 * (chi + chi.T))
    assert mu.min() > -1.0 and mu.max() <= 1e-12
    e = np.linalg.eigvalsh(0.5 * (screening.epsinv_dense(tiny_chib)
                                  + screening.epsinv_dense(tiny_chib).T))
    assert e.min() > 0.0 and e.max() <= 1.0 + 1e-12


@pytest.mark.parametrize("kind", screening.KINDS)
def test_full_rank_pdep_form_is_dense(kind, tiny_oracle, tiny_chib):
    b, _, _ = tiny_oracle
    n = tiny_chib.shape[0]
    lam, vec = pdep_reference(tiny_chib, n)
    rng = np.random.default_rng(5)
    f = rng.standard_normal((3, n))
    dense = {"chibar": screening.chibar_dyson, "epsinv": screening.epsinv_dense,
             "wp": lambda c: screening.wp_dense(b, c)}[kind](tiny_chib)
    out = screening.pdep_screening(kind, lam, vec, f, b.sqrt_coulomb())
    np.testing.assert_allclose(out, f @ dense.T, atol=1e-11 * np.abs(f @ dense.T).max())


def test_planted_dyson_sign_is_caught(monkeypatch, free7):
    b, chib, lam = free7
    monkeypatch.setattr(screening, "chibar_dyson",
                        lambda c: np.linalg.solve(np.eye(c.shape[0]) + c, c))
    chi = screening.chibar_dyson(chib)
    assert np.abs(chi - np.diag(lam / (1.0 - lam))).max() > 1e-3 * np.abs(lam).max()

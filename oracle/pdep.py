"""Dense symmetrised chi0bar at omega = 0 and its eigendecomposition.

Test infrastructure (see ``oracle/__init__``).

* ``chi0bar_dense``: the Adler-Wiser sum over states (Eq. AdlerWiser) at
  omega = 0, Gamma only, with the Brillouin-zone integral replaced by 1/Omega
  (one k point) and the oscillator strengths of Eq. (oscillator) taken as
  pair-density coefficients <e_G | psi_v psi_c> over the PDEP sphere
  (G != 0, the body of Table limitqchi0).  For real orbitals the two
  resonant denominators coincide and
      chi0_GG' = 4 sum_{v occ} sum_{c empty} p_vc(G) p_vc(G') / (eps_v - eps_c),
      chi0bar  = v^{1/2} chi0 v^{1/2},   v^{1/2}(G) = sqrt(4 pi)/|G|.
  The factor 4 is 2 (spin) x 2 (the c.c. term of Eq. deltani).
* ``pdep_reference``: its n_pdep most negative eigenpairs (ascending), the
  PDEP basis of Eq. (eigendecompzerofreq).
* ``free_electron_chi0bar``: the V = 0 closed form, diagonal in G:
      lambda(G) = 16 pi / (Omega |G|^2) sum_{k occ, k+G in S, not occ} 1/(eps_k - eps_{k+G}),
  eps_k = |k|^2 / 2, valid when the occupied set is a closed shell.
* Imaginary frequencies (argument nu): at omega = i nu the two resonant
  denominators of Eq. AdlerWiser add to
      1/(eps_v - eps_c - i nu) + 1/(eps_v - eps_c + i nu)
          = 2 (eps_v - eps_c) / ((eps_v - eps_c)^2 + nu^2),
  so every 1/(eps_v - eps_c) above becomes (eps_v - eps_c)/((eps_v - eps_c)^2 + nu^2)
  (nu = 0 gives the static forms).
"""
from __future__ import annotations

import numpy as np

from .basis import Basis
from .hamiltonian import KSStates
from .response import occupied_grid


def pair_coefficients(basis: Basis, u_occ, u_emp_block):
    """p_vc = <e_G | psi_v psi_c> (G != 0) for a block of empty states.

    Returns shape (N_occ, n_block, 2 n_half).
    """
    nocc = u_occ.shape[0]
    nb = u_emp_block.shape[0]
    prod = (u_occ[:, None] * u_emp_block[None, :]) / np.sqrt(basis.omega)
    c = basis.grid_to_coeffs(prod.reshape((nocc * nb,) + basis.grid))
    return c[:, :-1].reshape(nocc, nb, basis.n_pdep_dim)


def resolvent_weight(den, nu: float):
    """Weight of one (v, c) pair in the Adler-Wiser sum at omega = i nu (Sec.
    II B, Eq. AdlerWiser): with den = eps_v - eps_c, each of its two
    denominators contributes Re 1/(den +- i nu) = den / (den^2 + nu^2)."""
    return den / (den * den + nu * nu)


def chi0bar_dense(basis: Basis, ks: KSStates, block: int = 64, nu: float = 0.0) -> np.ndarray:
    """Dense chi0bar(i nu) on the PDEP sphere, shape (2 n_half, 2 n_half)."""
    nocc = ks.n_occ
    u_occ = occupied_grid(basis, ks)
    dim = basis.n_pdep_dim
    chi0 = np.zeros((dim, dim))
    ev = ks.eps[:nocc]
    for c0 in range(nocc, basis.n_pw, block):
        c1 = min(basis.n_pw, c0 + block)
        u_emp = basis.coeffs_to_grid(ks.C[:, c0:c1].T)
        p = pair_coefficients(basis, u_occ, u_emp)               # (nocc, nb, dim)
        den = ev[:, None] - ks.eps[c0:c1][None, :]              # eps_v - eps_c
        pw = p * resolvent_weight(den, nu)[:, :, None]
        chi0 += 4.0 * np.einsum("vcg,vch->gh", pw, p, optimize=True)
    vh = basis.sqrt_coulomb()
    chib = vh[:, None] * chi0 * vh[None, :]
    return chib


def pdep_reference(chib: np.ndarray, n_pdep: int):
    """The n_pdep most negative eigenpairs of chi0bar (ascending)."""
    sym = 0.5 * (chib + chib.T)
    lam, vec = np.linalg.eigh(sym)
    return lam[:n_pdep], vec[:, :n_pdep]


def free_electron_chi0bar(basis: Basis, n_occ: int, nu: float = 0.0) -> np.ndarray:
    """Closed-form eigenvalue of chi0bar(i nu) per PDEP component for V = 0.

    Requires the n_occ lowest plane waves to be a closed shell.
    Returns an array of length 2 n_half (both real components of G_k).
    """
    full = basis.full
    L = np.asarray(basis.cell)
    g2 = basis.g2_full
    order = np.argsort(g2, kind="stable")
    occ_set = set(map(tuple, full[order[:n_occ]]))
    if n_occ < len(order) and np.isclose(g2[order[n_occ - 1]], g2[order[n_occ]]):
        raise ValueError("n_occ is not a closed shell")
    sphere_set = set(map(tuple, full))
    lam = np.zeros(basis.n_half)
    for k_idx, G in enumerate(basis.half):
        s = 0.0
        for k in occ_set:
            q = (k[0] + G[0], k[1] + G[1], k[2] + G[2])
            if q in sphere_set and q not in occ_set:
                ek = 0.5 * np.sum((2 * np.pi * np.asarray(k) / L) ** 2)
                eq = 0.5 * np.sum((2 * np.pi * np.asarray(q) / L) ** 2)
                s += (ek - eq) / ((ek - eq) ** 2 + nu * nu)
        G2 = np.sum((2 * np.pi * G / L) ** 2)
        lam[k_idx] = 16.0 * np.pi / (basis.omega * G2) * s
    return np.repeat(lam, 2)

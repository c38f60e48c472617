"""Reducible polarizability, inverse dielectric matrix and W_p at omega = 0.

Test infrastructure (see ``oracle/__init__``).

What the PDEP eigenpairs are for (Sec. II A): once chi0bar is known, the
symmetrised reducible polarizability follows from the RPA Dyson equation
    chibar = (1 - chi0bar)^{-1} chi0bar                 (Eq. linearalgebrachichi0)
the symmetrised inverse dielectric matrix from
    epsbar^{-1} = 1 + chibar                            (Eq. epsilonandchi)
and the correlation part of the screened interaction from
    W^p_GG' = v^{1/2}(G) chibar_GG' v^{1/2}(G')         (Eq. Wpnondiag)
with v^{1/2}(G) = sqrt(4 pi)/|G| in Hartree units.  (Eq. Wpnondiag prints
chibar/(|G||G'|) with the 4 pi e^2 of the Coulomb factors absorbed; with it
written out, W = v + W^p = epsbar^{-1}-screened v, the form used here.)
chibar and chi0bar share their eigenvectors (Sec. II A after Eq.
eigendecompanyfreq, and Sec. II C), so in the PDEP basis {phi_i, lambda_i} of Eq.
(eigendecompzerofreq) at omega = 0
    chibar ~= sum_i phi_i lambda_i / (1 - lambda_i) phi_i^T,
which is what ``pdep_screening`` applies.  The dense functions take the
whole chi0bar matrix and are the definition; ``pdep_screening`` is the
low-rank form the GPU library computes.

Frequency dependence (Sec. II B, Eqs. finalB and Bfinal): the body of chi0bar
at imaginary frequency i nu in the PDEP basis,
    B_ij(i nu) = phi_i^T chi0bar(i nu) phi_j,
and its RPA screening Lambda(i nu) = (1 - B)^{-1} B (Eq. Bfinal without the
head and wings, which lie outside the PDEP sphere).

Functions
* ``pdep_body``         B(i nu) = Phi^T chi0bar(i nu) Phi from a dense chi0bar(i nu).
* ``lambda_body``       (1 - B)^{-1} B by a linear solve.
* ``chibar_dyson``      dense (1 - chi0bar)^{-1} chi0bar by a linear solve.
* ``epsinv_dense``      dense 1 + chibar.
* ``wp_dense``          dense v^{1/2} chibar v^{1/2}.
* ``pdep_screening``    the rank-n_pdep operator applied to vectors.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis

KINDS = ("chibar", "epsinv", "wp")


def chibar_dyson(chi0bar: np.ndarray) -> np.ndarray:
    """(1 - chi0bar)^{-1} chi0bar, Eq. (linearalgebrachichi0), by np.linalg.solve."""
    n = chi0bar.shape[0]
    return np.linalg.solve(np.eye(n) - chi0bar, chi0bar)


def epsinv_dense(chi0bar: np.ndarray) -> np.ndarray:
    """epsbar^{-1} = 1 + chibar, Eq. (epsilonandchi)."""
    return np.eye(chi0bar.shape[0]) + chibar_dyson(chi0bar)


def wp_dense(basis: Basis, chi0bar: np.ndarray) -> np.ndarray:
    """W^p = v^{1/2} chibar v^{1/2} on the PDEP sphere, Eq. (Wpnondiag)."""
    vh = basis.sqrt_coulomb()
    return vh[:, None] * chibar_dyson(chi0bar) * vh[None, :]


def pdep_screening(kind: str, lam, vecs, f, sqrt_coulomb=None) -> np.ndarray:
    """Apply the PDEP (rank n_pdep) form of chibar, epsbar^{-1} or W^p.

    lam [n_pdep] and vecs [dim, n_pdep] are eigenpairs of chi0bar (the
    columns orthonormal); f [n, dim] holds n vectors on the PDEP sphere.
    Returns [n, dim]:
      chibar: Phi diag(lambda/(1-lambda)) Phi^T f
      epsinv: f + Phi diag(lambda/(1-lambda)) Phi^T f
      wp:     D Phi diag(lambda/(1-lambda)) Phi^T D f,  D = diag(sqrt(4 pi)/|G|)
    """
    if kind not in KINDS:
        raise ValueError(kind)
    lam = np.asarray(lam, dtype=np.float64)
    vecs = np.asarray(vecs, dtype=np.float64)
    f = np.atleast_2d(np.asarray(f, dtype=np.float64))
    g = lam / (1.0 - lam)
    x = f * sqrt_coulomb[None, :] if kind == "wp" else f
    out = ((x @ vecs) * g[None, :]) @ vecs.T
    if kind == "wp":
        out = out * sqrt_coulomb[None, :]
    if kind == "epsinv":
        out = out + f
    return out


def pdep_body(chi0bar_nu: np.ndarray, vecs) -> np.ndarray:
    """B = Phi^T chi0bar(i nu) Phi for PDEP vectors vecs [dim, n_pdep] (Eq. finalB)."""
    vecs = np.asarray(vecs, dtype=np.float64)
    return vecs.T @ chi0bar_nu @ vecs


def lambda_body(B: np.ndarray) -> np.ndarray:
    """Lambda = (1 - B)^{-1} B (Eq. Bfinal, body only), by np.linalg.solve."""
    return np.linalg.solve(np.eye(B.shape[0]) - B, B)

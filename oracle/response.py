"""Sternheimer solutions, density response and chi0bar applied to vectors.

Test infrastructure (see ``oracle/__init__``).

Sec. II C of the paper.  For a perturbing potential dV and each occupied
state v the Sternheimer equation (Eq. stern)
    (H - eps_v) P_c dpsi_v = - P_c dV psi_v,     P_c = 1 - sum_v |v><v|,
is solved for P_c dpsi_v, here two independent ways:
  * ``sternheimer_sos``: expansion over every empty state c of the finite
    basis, P_c dpsi_v = sum_c |c> <c|dV|v> / (eps_v - eps_c)  (the
    completeness argument the paper uses to drop virtual states);
  * ``sternheimer_cg``: plain conjugate gradients on P_c (H - eps_v) P_c,
    restricted to range(P_c), with the dense H.
The density response (Eq. deltani), spin-unpolarised with real orbitals, is
    dn(r) = 2 (spin) * sum_v [dpsi_v* psi_v + c.c.] = 4 sum_v psi_v(r) dpsi_v(r).
chi0bar applied to a PDEP vector phi (Eqs. symmoperator, chiisamatrixinpdep,
Hartree units, e^2 = 1): the perturbation is dV = v^{1/2} phi, i.e.
dV(G) = sqrt(4 pi)/|G| phi(G) for G != 0, and (chi0bar phi)(G) =
sqrt(4 pi)/|G| dn(G), dn(G) the orthonormal-basis coefficient of dn.

Grid normalisation: psi_v(r) = Omega^{-1/2} u_v(r), u_v = coeffs_to_grid(c_v).
"""
from __future__ import annotations

import numpy as np

from .basis import Basis
from .hamiltonian import KSStates


def occupied_grid(basis: Basis, ks: KSStates):
    """u_v(r) for the occupied states, shape (N_occ, *grid)."""
    return basis.coeffs_to_grid(ks.C[:, : ks.n_occ].T)


def perturbation_projections(basis: Basis, u_occ, dv_r):
    """<e_G | dV psi_v> for all v, shape (N_occ, N_pw) (full sphere incl. G=0)."""
    prod = np.asarray(dv_r)[None] * u_occ           # Omega^{1/2} (dV psi_v)
    return basis.grid_to_coeffs(prod)


def sternheimer_sos(basis: Basis, ks: KSStates, dv_r, u_occ=None):
    """P_c dpsi_v for one dV(r) by the sum over empty states; (N_occ, N_pw)."""
    if u_occ is None:
        u_occ = occupied_grid(basis, ks)
    nocc = ks.n_occ
    w = perturbation_projections(basis, u_occ, dv_r)          # (nocc, npw)
    Ce = ks.C[:, nocc:]                                       # empty states
    ee = ks.eps[nocc:]
    ev = ks.eps[:nocc]
    proj = Ce.T @ w.T                                         # <c|dV|v>, (nemp, nocc)
    coef = proj / (ev[None, :] - ee[:, None])
    return (Ce @ coef).T


def sternheimer_cg(basis: Basis, ks: KSStates, h, dv_r, tol=1e-12, max_iter=5000,
                   u_occ=None, states=None):
    """P_c dpsi_v by CG on P_c (H - eps_v) P_c x = -P_c dV psi_v; (N_occ, N_pw).

    h is the dense Hamiltonian of the unperturbed system (dense_hamiltonian).
    states (optional) restricts the solves to those occupied indices; the
    other rows of the result stay zero.
    Returns (dpsi, iterations, relative residuals).
    """
    if u_occ is None:
        u_occ = occupied_grid(basis, ks)
    nocc = ks.n_occ
    Co = ks.C[:, :nocc]

    def pc(y):
        return y - Co @ (Co.T @ y)

    w = perturbation_projections(basis, u_occ, dv_r)
    out = np.zeros((nocc, basis.n_pw))
    its = np.zeros(nocc, dtype=int)
    res = np.zeros(nocc)
    for v in (range(nocc) if states is None else states):
        b = -pc(w[v])
        bn = np.linalg.norm(b)
        x = np.zeros_like(b)
        if bn == 0.0:
            continue
        r = b.copy()
        p = r.copy()
        rr = r @ r
        k = 0
        while k < max_iter and np.sqrt(rr) > tol * bn:
            ap = pc(h @ p - ks.eps[v] * p)
            alpha = rr / (p @ ap)
            x += alpha * p
            r -= alpha * ap
            rr_new = r @ r
            p = r + (rr_new / rr) * p
            rr = rr_new
            k += 1
        x = pc(x)
        out[v] = x
        its[v] = k
        res[v] = np.linalg.norm(b - pc(h @ x - ks.eps[v] * x)) / bn
    return out, its, res


def density_response(basis: Basis, u_occ, dpsi):
    """dn(r) = 4 sum_v psi_v dpsi_v = (4/Omega) sum_v u_v du_v  (Eq. deltani)."""
    du = basis.coeffs_to_grid(dpsi)                 # (nocc, *grid)
    return (4.0 / basis.omega) * np.sum(u_occ * du, axis=0)


def chi0bar_apply(basis: Basis, ks: KSStates, phi, u_occ=None, return_dn=False):
    """chi0bar phi for PDEP vectors phi, shape (n, 2 n_half), by sum over states.

    Returns chi0bar phi (n, 2 n_half) and optionally dn(r) (n, *grid).
    """
    phi = np.atleast_2d(np.asarray(phi, dtype=np.float64))
    if u_occ is None:
        u_occ = occupied_grid(basis, ks)
    vh = basis.sqrt_coulomb()
    out = np.empty_like(phi)
    dns = []
    for j in range(phi.shape[0]):
        x = np.concatenate([vh * phi[j], [0.0]])             # v^{1/2} phi, G=0 empty
        dv = basis.coeffs_to_grid(x) / np.sqrt(basis.omega)  # dV(r), Ha
        dpsi = sternheimer_sos(basis, ks, dv, u_occ)
        dn = density_response(basis, u_occ, dpsi)
        dn_c = basis.grid_to_coeffs(np.sqrt(basis.omega) * dn)
        out[j] = vh * dn_c[:-1]
        dns.append(dn)
    if return_dn:
        return out, np.asarray(dns)
    return out


def density_from_states(basis: Basis, ks: KSStates):
    """n(r) = 2 sum_v |psi_v(r)|^2 (spin-unpolarised)."""
    u = occupied_grid(basis, ks)
    return (2.0 / basis.omega) * np.sum(u * u, axis=0)

"""Lanczos chains of the deflated Hamiltonian and the resolvent they give.

Test infrastructure (see ``oracle/__init__``).

Sec. II D of the paper.  The conduction-manifold matrix element
    M_c,LR(omega) = <L| P_c O(omega) P_c |R>,  O(omega) = -(H - omega)^{-1}
(Eqs. MC, Odef) is written with the deflated Hamiltonian H~ = P_c H P_c as
    M_c,LR(omega) = - <L| (H~ - omega)^{-1} |R>                  (Eq. MCdef)
and evaluated from a Lanczos chain started on R: q_1 = R, then
    alpha_n = <q_n|H~|q_n>,
    beta_{n+1} q_{n+1} = (H~ - alpha_n) q_n - beta_n q_{n-1},  beta_{n+1} = norm,
the tridiagonal T of the alphas and betas is diagonalised, D = U^T T U, and
    M_c,LR(omega) = - sum_{n1,n2} <L|q_n1> U_{n1 n2} U_{1 n2} / (d_n2 - omega)
                                                                  (Eq. MCfinal)
whose coefficients do not depend on omega.

Reading: the paper's q_1 = R presumes a normalised R inside range(P_c); here
q_1 = P_c R / ||P_c R|| and M carries the factor ||P_c R||, so that M equals
Eq. MCdef for any R.  The recursion is the paper's three-term one, without
reorthogonalisation.

Functions
* ``deflated_hamiltonian``  dense P_c H P_c.
* ``lanczos_chain``         alpha [K], beta [K] (beta[0] = ||P_c R||), Q [K, dim].
* ``lanczos_poles_weights`` d [K] and the omega-independent weights
                            w[l, n2] = ||P_c R|| sum_n1 <L_l|q_n1> U_{n1 n2} U_{1 n2},
                            so that M_c(omega) = sum_n2 w[l, n2] / (omega - d_n2).
* ``lanczos_resolvent``     M_c(omega) from them (Eq. MCfinal).
* ``resolvent_sos``         the exact M_c(omega) = -sum_c <L|c><c|R> / (eps_c - omega)
                            over the empty states of the finite basis.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import KSStates


def deflated_hamiltonian(h: np.ndarray, ks: KSStates) -> np.ndarray:
    """P_c H P_c with P_c = 1 - sum_v |v><v| over the occupied states."""
    v = ks.C[:, : ks.n_occ]
    pc = np.eye(h.shape[0]) - v @ v.T
    return pc @ h @ pc


def lanczos_chain(hd: np.ndarray, r: np.ndarray, n_steps: int, pc=None):
    """Three-term Lanczos recursion on hd started on P_c r.

    pc: optional P_c as a function of a vector (else r is used as given).
    Returns alpha [n_steps], beta [n_steps] with beta[0] = ||P_c r|| and
    beta[k] (k >= 1) the off-diagonal T[k-1, k], and Q [n_steps, dim].  A
    chain that reaches an invariant subspace (beta_{n+1} at or below 1e-12
    ||H~ q_n||) stops; its remaining entries are zero.  A start vector with
    ||P_c r|| at or below 1e-12 ||r|| gives an empty chain.
    """
    r = np.asarray(r, dtype=np.float64)
    q0 = pc(r) if pc is not None else r.copy()
    b0 = float(np.linalg.norm(q0))
    if b0 <= 1e-12 * float(np.linalg.norm(r)):
        b0 = 0.0                      # start vector inside the occupied space
    dim = q0.shape[0]
    alpha = np.zeros(n_steps)
    beta = np.zeros(n_steps)
    Q = np.zeros((n_steps, dim))
    beta[0] = b0
    if b0 == 0.0:
        return alpha, beta, Q
    Q[0] = q0 / b0
    q_prev = np.zeros(dim)
    b_prev = 0.0
    for n in range(n_steps):
        w = hd @ Q[n]
        hn = float(np.linalg.norm(w))
        alpha[n] = Q[n] @ w
        w = w - alpha[n] * Q[n] - b_prev * q_prev
        if n + 1 == n_steps:
            break
        b = float(np.linalg.norm(w))
        if b <= 1e-12 * hn:
            break
        beta[n + 1] = b
        Q[n + 1] = w / b
        q_prev, b_prev = Q[n], b
    return alpha, beta, Q


def tridiagonal(alpha, beta) -> np.ndarray:
    """T with alpha on the diagonal and beta[1:] on the off-diagonals."""
    k = len(alpha)
    t = np.diag(np.asarray(alpha, dtype=np.float64))
    for i in range(1, k):
        t[i - 1, i] = t[i, i - 1] = beta[i]
    return t


def lanczos_poles_weights(alpha, beta, Q, L):
    """Poles d [K] and weights w [n_L, K] of Eq. MCfinal for the rows of L."""
    d, u = np.linalg.eigh(tridiagonal(alpha, beta))
    lq = np.atleast_2d(L) @ Q.T                       # <L_l | q_n1>, [n_L, K]
    w = beta[0] * (lq @ u) * u[0][None, :]
    return d, w


def lanczos_resolvent(d, w, omegas):
    """M_c(omega) = sum_n w[l, n] / (omega - d_n) for every omega; [n_L, n_omega]."""
    om = np.asarray(omegas)
    return np.einsum("ln,nw->lw", w, 1.0 / (om[None, :] - d[:, None]))


def resolvent_sos(ks: KSStates, L, R, omegas):
    """Exact M_c(omega) = -sum_c <L|c><c|R> / (eps_c - omega), c empty; [n_L, n_omega]."""
    ce = ks.C[:, ks.n_occ:]
    ee = ks.eps[ks.n_occ:]
    lc = np.atleast_2d(L) @ ce                         # [n_L, n_emp]
    cr = ce.T @ np.asarray(R)                          # [n_emp]
    om = np.asarray(omegas)
    return -np.einsum("lc,c,cw->lw", lc, cr, 1.0 / (ee[:, None] - om[None, :]))

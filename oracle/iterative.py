"""Large-system routes of the oracle: Kohn-Sham states by a Lanczos
eigensolver on the grid-applied H, and Sternheimer solves by preconditioned
conjugate gradients with H applied by grid products.

Test infrastructure (see ``oracle/__init__``).

The dense routes of ``hamiltonian`` and ``response`` hold N_pw x N_pw
matrices; at the 64x64x192 interface (49 095 plane waves) those no longer
fit, and the 64^3 systems of the uneven batch (16 375) are slow.  The
routes here reach the same results without any dense matrix:

* ``apply_h`` evaluates H x = 1/2|G|^2 x + <e_G|V u> for a block of vectors
  with real-to-complex FFTs (the formula of ``hamiltonian.apply_hamiltonian_grid``
  written for many vectors at once);
* ``ks_states_lanczos`` takes the lowest eigenpairs of that operator with
  ARPACK's implicitly restarted Lanczos (scipy ``eigsh``), the Kohn-Sham
  states of Eq. secEqforHKS for a local potential;
* ``sternheimer_pcg`` solves Eq. stern, P_c (H - eps_v) P_c x = -P_c dV psi_v
  on range(P_c), for many occupied states at once by conjugate gradients
  preconditioned with P_c K P_c, K(G) = 1 / max(1, (|G|^2/2) / T_v) (a
  diagonal kinetic-energy preconditioner, T_v the kinetic energy of psi_v;
  the paper asks for a preconditioned CG without naming one, and a
  preconditioner changes the iteration count, not the solution);
* ``chi0bar_apply_pcg`` is ``response.chi0bar_apply`` with the Sternheimer
  solutions from ``sternheimer_pcg`` (Eqs. deltani, chiisamatrixinpdep).

Pinned in tests/test_oracle_iterative.py against the dense routes on small
systems (eigenpairs against ``ks_states``; solutions and chi0bar phi against
the sum over all empty states).
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft
from scipy.sparse.linalg import LinearOperator, eigsh

from .basis import Basis
from .hamiltonian import KSStates

_WORKERS = os.cpu_count() or 1


def _half_index(basis: Basis):
    """Grid positions of the half-space members on the real-FFT layout
    (n3 >= 0 for every half-space member), their n3 = 0 mirrors, and the
    positions of those mirrors."""
    N = basis.grid
    h = basis.half
    pos = tuple(h[:, a] % N[a] for a in range(3))
    m0 = np.nonzero(h[:, 2] == 0)[0]              # members on the n3 = 0 plane
    mpos = tuple((-h[m0, a]) % N[a] for a in range(3))
    return pos, m0, mpos


def to_grid(basis: Basis, X, chunk: int = 32):
    """u(r) = sum_G c(G) e^{iG.r} for the rows of X (real layout), by
    complex-to-real FFTs over the n3 >= 0 half of the grid; shape (n, *grid)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    N1, N2, N3 = basis.grid
    nh = basis.n_half
    pos, m0, mpos = _half_index(basis)
    s = 1.0 / np.sqrt(2.0)
    out = np.empty((X.shape[0],) + basis.grid)
    for a in range(0, X.shape[0], chunk):
        xb = X[a:a + chunk]
        c = s * (xb[:, 0:2 * nh:2] + 1j * xb[:, 1:2 * nh:2])     # c(G_k), k < nh
        A = np.zeros((xb.shape[0], N1, N2, N3 // 2 + 1), dtype=np.complex128)
        A[(slice(None),) + pos] = c
        A[(slice(None),) + mpos] = np.conj(c[:, m0])             # c(-G) = conj c(G)
        A[:, 0, 0, 0] = xb[:, 2 * nh]
        out[a:a + chunk] = sfft.irfftn(A, s=basis.grid, axes=(1, 2, 3), workers=_WORKERS) * basis.n_r
    return out


def from_grid(basis: Basis, U, chunk: int = 32):
    """Real-layout coefficients c(G) = FFT[u](G) / N_r of real grids U
    (shape (n, *grid)) on the sphere; inverse of ``to_grid`` on band-limited
    input."""
    U = np.asarray(U, dtype=np.float64).reshape((-1,) + basis.grid)
    nh = basis.n_half
    pos, _, _ = _half_index(basis)
    out = np.empty((U.shape[0], basis.n_pw))
    for a in range(0, U.shape[0], chunk):
        F = sfft.rfftn(U[a:a + chunk], axes=(1, 2, 3), workers=_WORKERS) / basis.n_r
        c = F[(slice(None),) + pos]
        out[a:a + chunk, 0:2 * nh:2] = np.sqrt(2.0) * c.real
        out[a:a + chunk, 1:2 * nh:2] = np.sqrt(2.0) * c.imag
        out[a:a + chunk, 2 * nh] = F[:, 0, 0, 0].real
    return out


def apply_h(basis: Basis, v_r, X, chunk: int = 32):
    """H x = 1/2 |G|^2 x + <e_G | V u> for the rows of X, u = to_grid(x)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    V = np.asarray(v_r, dtype=np.float64).reshape(basis.grid)
    out = np.empty_like(X)
    for a in range(0, X.shape[0], chunk):
        u = to_grid(basis, X[a:a + chunk], chunk)
        out[a:a + chunk] = 0.5 * basis.g2_real[None] * X[a:a + chunk] + from_grid(basis, V[None] * u,
                                                                                  chunk)
    return out


def ks_states_lanczos(basis: Basis, v_r, n_occ: int, n_states: int | None = None,
                      tol: float = 1e-14) -> KSStates:
    """The n_states (default n_occ + 1) lowest eigenpairs of H by ARPACK
    Lanczos on H + s, s = 1 - min V (all eigenvalues >= 1, so ARPACK's
    relative tolerance is an absolute one of the same size).  C holds only
    those states (N_pw x n_states)."""
    k = int(n_occ + 1 if n_states is None else n_states)
    shift = 1.0 - float(np.min(v_r))
    n = basis.n_pw

    def mv(x):
        return apply_h(basis, v_r, x[None])[0] + shift * x

    def mm(X):
        return (apply_h(basis, v_r, X.T) + shift * X.T).T

    op = LinearOperator((n, n), matvec=mv, matmat=mm, dtype=np.float64)
    w, C = eigsh(op, k=k, which="SA", tol=tol, ncv=min(n - 1, 2 * k + 40))
    order = np.argsort(w)
    return KSStates(eps=w[order] - shift, C=C[:, order], n_occ=int(n_occ))


def kinetic_preconditioner(basis: Basis, ks: KSStates):
    """K_v(G) = 1 / max(1, (|G|^2/2) / T_v) per occupied state, T_v =
    sum_G |G|^2/2 |c_v(G)|^2 (floored at 0.1 Ha); shape (n_occ, N_pw)."""
    Co = ks.C[:, : ks.n_occ]
    t = 0.5 * basis.g2_real
    tv = np.maximum(t @ (Co * Co), 0.1)
    return 1.0 / np.maximum(1.0, t[None, :] / tv[:, None])


def sternheimer_pcg(basis: Basis, ks: KSStates, v_r, dv_r, states=None, tol: float = 1e-12,
                    max_iter: int = 20000, u_occ=None):
    """P_c dpsi_v for one perturbing potential dV(r) (Eq. stern) by
    preconditioned CG, all listed occupied states at once (each its own CG).

    Solves P_c (H - eps_v) P_c x = b, b = -P_c dV psi_v, on range(P_c) with
    the preconditioner z = P_c K_v r; stops when ||r|| <= tol ||b|| for the
    CG recursion's residual r.  Returns (dpsi (n_occ, N_pw) with zero rows
    for unlisted states, iterations, relative residuals ||b - A x|| / ||b||
    recomputed from x)."""
    nocc = ks.n_occ
    Co = ks.C[:, :nocc]
    idx = np.arange(nocc) if states is None else np.asarray(states, dtype=int)
    eps = ks.eps[idx]
    if u_occ is None:
        u_occ = to_grid(basis, Co[:, idx].T)
    else:
        u_occ = np.asarray(u_occ)[idx]
    K = kinetic_preconditioner(basis, ks)[idx]

    def pc(Y):                                   # rows of Y projected on range(P_c)
        return Y - (Y @ Co) @ Co.T

    def op(Y, e):
        return pc(apply_h(basis, v_r, Y) - e[:, None] * Y)

    b = -pc(from_grid(basis, np.asarray(dv_r).reshape(basis.grid)[None] * u_occ))
    bn = np.linalg.norm(b, axis=1)
    x = np.zeros_like(b)
    r = b.copy()
    z = pc(K * r)
    p = z.copy()
    rz = np.sum(r * z, axis=1)
    its = np.zeros(len(idx), dtype=int)
    act = np.nonzero(bn > 0.0)[0]
    k = 0
    while act.size and k < max_iter:
        ap = op(p[act], eps[act])
        alpha = rz[act] / np.sum(p[act] * ap, axis=1)
        x[act] += alpha[:, None] * p[act]
        r[act] -= alpha[:, None] * ap
        its[act] += 1
        rn = np.linalg.norm(r[act], axis=1)
        done = rn <= tol * bn[act]
        z_a = pc(K[act] * r[act])
        rz_new = np.sum(r[act] * z_a, axis=1)
        beta = rz_new / rz[act]
        p[act] = z_a + beta[:, None] * p[act]
        rz[act] = rz_new
        act = act[~done]
        k += 1
    x = pc(x)
    res = np.zeros(len(idx))
    nz = bn > 0.0
    if np.any(nz):
        res[nz] = np.linalg.norm(b[nz] - op(x[nz], eps[nz]), axis=1) / bn[nz]
    out = np.zeros((nocc, basis.n_pw))
    out[idx] = x
    return out, its, res


def chi0bar_apply_pcg(basis: Basis, ks: KSStates, v_r, phi, tol: float = 1e-12,
                      return_dn: bool = False):
    """chi0bar phi for PDEP vectors phi (n, 2 n_half), with every Sternheimer
    solution from ``sternheimer_pcg`` over all occupied states: dV = v^{1/2}
    phi on the grid, dn(r) = 4 sum_v psi_v dpsi_v (Eq. deltani), chi0bar phi
    = v^{1/2} dn(G) (Eq. chiisamatrixinpdep).  Returns chi0bar phi and, with
    return_dn, dn(r) (n, *grid)."""
    phi = np.atleast_2d(np.asarray(phi, dtype=np.float64))
    Co = ks.C[:, : ks.n_occ]
    u_occ = to_grid(basis, Co.T)
    vh = basis.sqrt_coulomb()
    out = np.empty_like(phi)
    dns = []
    for j in range(phi.shape[0]):
        xg = np.concatenate([vh * phi[j], [0.0]])
        dv = to_grid(basis, xg[None])[0] / np.sqrt(basis.omega)
        dpsi, _, _ = sternheimer_pcg(basis, ks, v_r, dv, tol=tol, u_occ=u_occ)
        dn = (4.0 / basis.omega) * np.einsum("vxyz,vxyz->xyz", u_occ, to_grid(basis, dpsi))
        dn_c = from_grid(basis, np.sqrt(basis.omega) * dn[None])[0]
        out[j] = vh * dn_c[:-1]
        dns.append(dn)
    if return_dn:
        return out, np.asarray(dns)
    return out

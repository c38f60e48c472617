"""Dense Kohn-Sham Hamiltonian of a local potential and its eigenpairs.

Test infrastructure (see ``oracle/__init__``).

Stands in for the ground-state step of Sec. II (Eq. secEqforHKS): for the
synthetic systems H = -1/2 nabla^2 + V(r), with V local.  In the orthonormal
plane-wave basis of the sphere
    H_GG' = 1/2 |G|^2 delta_GG' + V(G - G'),
    V(g)  = N_r^{-1} sum_k V(r_k) exp(-i g.r_k)   (the grid DFT of V).
The complex matrix is rotated to the real layout, H_real = U^H H U, and
diagonalised with LAPACK.  Occupations are integer: the N_occ lowest states
are occupied (a gap is required, as for the insulators of the paper).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .basis import Basis


def potential_fourier(basis: Basis, v_r):
    """V(g) on the grid's DFT index set: fftn(V)/N_r."""
    return np.fft.fftn(np.asarray(v_r, dtype=np.float64)) / basis.n_r


def dense_hamiltonian(basis: Basis, v_r) -> np.ndarray:
    """Real symmetric H in the real-coefficient layout, shape (N_pw, N_pw)."""
    vg = potential_fourier(basis, v_r)
    full = basis.full
    N1, N2, N3 = basis.grid
    # V(G_a - G_b) for all pairs of the full list, via a flat grid index
    flat = (full[:, 0][:, None] - full[:, 0][None, :]) % N1
    flat = flat * N2 + (full[:, 1][:, None] - full[:, 1][None, :]) % N2
    flat = flat * N3 + (full[:, 2][:, None] - full[:, 2][None, :]) % N3
    hc = vg.ravel()[flat]
    del flat
    hc[np.diag_indices_from(hc)] += 0.5 * basis.g2_full
    # H_real = U^H Hc U, with U sparse
    t = basis.UH @ hc                     # (N_pw, N_pw) dense
    h = (basis.U.T @ t.T).T               # t @ U
    assert np.max(np.abs(h.imag)) <= 1e-12 * max(1.0, np.max(np.abs(h.real))), \
        "H is not real in the real layout"
    h = h.real
    return 0.5 * (h + h.T)


def apply_hamiltonian_grid(basis: Basis, v_r, x):
    """H x evaluated with grid products (independent of dense_hamiltonian).

    (H x)(G) = 1/2|G|^2 x(G) + [FFT(V u) / N_r](G),  u = coeffs_to_grid(x).
    """
    x = np.asarray(x, dtype=np.float64)
    u = basis.coeffs_to_grid(x)
    vx = basis.grid_to_coeffs(np.asarray(v_r)[None] * u.reshape((-1,) + basis.grid))
    return 0.5 * basis.g2_real * x + vx.reshape(x.shape)


@dataclass
class KSStates:
    eps: np.ndarray        # all eigenvalues, ascending (Ha)
    C: np.ndarray          # eigenvectors as columns, real layout (N_pw, N_pw)
    n_occ: int

    @property
    def gap(self) -> float:
        return float(self.eps[self.n_occ] - self.eps[self.n_occ - 1])


def ks_states(basis: Basis, v_r, n_occ: int) -> KSStates:
    """All eigenpairs of the dense H; the n_occ lowest are occupied."""
    h = dense_hamiltonian(basis, v_r)
    eps, C = np.linalg.eigh(h)
    return KSStates(eps=eps, C=C, n_occ=int(n_occ))

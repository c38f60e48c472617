"""Plane-wave sphere at Gamma and the real-coefficient vector layout.

Test infrastructure (see ``oracle/__init__``).

Follows Eq. (planewaveexpansionofwfc), Sec. II A: a function is expanded in
plane waves exp(iG.r) with 1/2|G|^2 <= E_cut.  Here the basis is
orthonormal on the cell: e_G(r) = Omega^{-1/2} exp(iG.r), so a real function
is f(r) = Omega^{-1/2} sum_G c(G) exp(iG.r) with c(-G) = conj c(G).

Conventions (identical to the C ABI header, written independently here):
  * reciprocal vectors G = 2 pi (n1/L1, n2/L2, n3/L3), n integer;
  * E_cut = 0 means "derive from the grid": r_i = (N_i - 1)/4 grid steps,
    E_cut = 1/2 (min_i 2 pi r_i / L_i)^2, which keeps every product of two
    sphere functions alias-free on the grid;
  * half space H+ = {n3 > 0} u {n3 = 0, n2 > 0} u {n3 = n2 = 0, n1 > 0},
    its sphere members sorted by (n3, n2, n1) ascending: G_0 .. G_{nh-1};
  * real vector of length N_pw = 2 nh + 1:
        x[2k] = sqrt2 Re c(G_k),  x[2k+1] = sqrt2 Im c(G_k),  x[2nh] = c(0),
    so the Euclidean dot product of two vectors is the L2 inner product;
  * a PDEP vector (no G = 0 component) is the first 2 nh entries.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def derived_ecut(grid, cell) -> float:
    """E_cut from the grid rule r_i = (N_i - 1)/4 (alias-free products)."""
    N = np.asarray(grid, dtype=np.float64)
    L = np.asarray(cell, dtype=np.float64)
    r = (N - 1.0) / 4.0
    gmax = np.min(2.0 * np.pi * r / L)
    return 0.5 * gmax * gmax


class Basis:
    """Sphere members, the complex<->real coefficient map and grid transforms."""

    def __init__(self, grid, cell, ecut: float = 0.0):
        self.grid = tuple(int(n) for n in grid)
        self.cell = tuple(float(l) for l in cell)
        self.omega = float(np.prod(self.cell))
        self.n_r = int(np.prod(self.grid))
        self.ecut = float(ecut) if ecut > 0 else derived_ecut(self.grid, self.cell)

        # all integer triples strictly inside the grid's Nyquist box
        rng = [np.arange(-((n - 1) // 2), (n - 1) // 2 + 1) for n in self.grid]
        n1, n2, n3 = np.meshgrid(*rng, indexing="ij")
        n1, n2, n3 = n1.ravel(), n2.ravel(), n3.ravel()
        L = self.cell
        gx = 2.0 * np.pi * n1 / L[0]
        gy = 2.0 * np.pi * n2 / L[1]
        gz = 2.0 * np.pi * n3 / L[2]
        inside = 0.5 * (gx * gx + gy * gy + gz * gz) <= self.ecut
        upper = (n3 > 0) | ((n3 == 0) & (n2 > 0)) | ((n3 == 0) & (n2 == 0) & (n1 > 0))
        sel = inside & upper
        h1, h2, h3 = n1[sel], n2[sel], n3[sel]
        order = np.lexsort((h1, h2, h3))          # primary n3, then n2, then n1
        self.half = np.stack([h1[order], h2[order], h3[order]], axis=1)
        self.n_half = self.half.shape[0]
        self.n_pw = 2 * self.n_half + 1
        self.n_pdep_dim = 2 * self.n_half
        self.n_sphere = int(inside.sum())
        assert self.n_sphere == self.n_pw, "sphere is not inversion symmetric"

        # complex "full" list: [G_0..G_{nh-1}, -G_0..-G_{nh-1}, 0]
        self.full = np.concatenate([self.half, -self.half, np.zeros((1, 3), dtype=int)])
        g = 2.0 * np.pi * self.full / np.asarray(self.cell)[None, :]
        self.g2_full = np.sum(g * g, axis=1)
        gh = 2.0 * np.pi * self.half / np.asarray(self.cell)[None, :]
        g2h = np.sum(gh * gh, axis=1)
        # |G|^2 per real component (both components of G_k, then G = 0)
        self.g2_real = np.concatenate([np.repeat(g2h, 2), [0.0]])
        # grid positions of the full list (n mod N)
        self.full_grid_index = tuple((self.full[:, a] % self.grid[a]) for a in range(3))

        # c_full = U x  (unitary, two entries per column)
        nh = self.n_half
        s = 1.0 / np.sqrt(2.0)
        rows, cols, vals = [], [], []
        for k in range(nh):
            rows += [k, nh + k, k, nh + k]
            cols += [2 * k, 2 * k, 2 * k + 1, 2 * k + 1]
            vals += [s, s, 1j * s, -1j * s]
        rows.append(2 * nh)
        cols.append(2 * nh)
        vals.append(1.0 + 0j)
        self.U = sp.csr_matrix((np.asarray(vals, dtype=np.complex128), (rows, cols)),
                               shape=(self.n_pw, self.n_pw))
        self.UH = self.U.conj().T.tocsr()

    # -- coefficient <-> grid ------------------------------------------------
    def to_complex(self, x):
        """Real layout (..., N_pw) -> complex coefficients on the full list."""
        x = np.asarray(x, dtype=np.float64)
        return (self.U @ x.reshape(-1, self.n_pw).T).T.reshape(x.shape[:-1] + (self.n_pw,))

    def to_real(self, c):
        """Complex coefficients on the full list -> real layout (imag checked)."""
        c = np.asarray(c, dtype=np.complex128)
        x = (self.UH @ c.reshape(-1, self.n_pw).T).T.reshape(c.shape)
        return x.real

    def coeffs_to_grid(self, x):
        """u(r_k) = sum_G c(G) exp(i G.r_k) for real-layout x, shape (..., N_pw).

        The physical function is Omega^{-1/2} u.
        """
        x = np.asarray(x, dtype=np.float64)
        lead = x.shape[:-1]
        c = self.to_complex(x).reshape(-1, self.n_pw)
        out = np.empty((c.shape[0],) + self.grid, dtype=np.float64)
        for i in range(c.shape[0]):
            A = np.zeros(self.grid, dtype=np.complex128)
            A[self.full_grid_index] = c[i]
            u = np.fft.ifftn(A) * self.n_r
            out[i] = u.real
        return out.reshape(lead + self.grid)

    def grid_to_coeffs(self, u):
        """Inverse of coeffs_to_grid on band-limited input: c(G) = FFT[u](G)/N_r.

        For a physical function f, grid_to_coeffs(Omega^{1/2} f) gives its
        coefficients in the orthonormal basis restricted to the sphere.
        """
        u = np.asarray(u, dtype=np.float64)
        lead = u.shape[:-3]
        uu = u.reshape((-1,) + self.grid)
        c = np.empty((uu.shape[0], self.n_pw), dtype=np.complex128)
        for i in range(uu.shape[0]):
            F = np.fft.fftn(uu[i]) / self.n_r
            c[i] = F[self.full_grid_index]
        return self.to_real(c).reshape(lead + (self.n_pw,))

    def sqrt_coulomb(self):
        """v^{1/2}(G) = sqrt(4 pi)/|G| per PDEP component (Eq. symmoperator, e^2 = 1)."""
        return np.sqrt(4.0 * np.pi) / np.sqrt(self.g2_real[:-1])

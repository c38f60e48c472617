"""Plain FP64 CPU oracle for the PDEP hot path (TEST INFRASTRUCTURE ONLY).

This package is the slow, obviously-correct reference that the CUDA
library is checked against.  It is test infrastructure: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA path; both consume the seeded
inputs of the ``synthetic`` package.

What it computes, in the paper's notation (Govoni & Galli, "Large scale
GW calculations"), Hartree atomic units, Gamma point, spin-unpolarised,
real orbitals:

* ``basis``       plane-wave sphere 1/2|G|^2 <= E_cut (Eq. planewaveexpansionofwfc)
                  and the real-coefficient vector layout shared with the C ABI.
* ``hamiltonian`` dense H_GG' = 1/2|G|^2 d_GG' + V(G-G') and its eigenpairs
                  (the Kohn-Sham states of Eq. secEqforHKS for a local potential).
* ``response``    Sternheimer solution of Eq. stern (by explicit sum over the
                  empty states of the finite basis, and by CG), the density
                  response of Eq. deltani, and chi0bar applied to PDEP vectors
                  (Eqs. symmoperator and chiisamatrixinpdep).
* ``pdep``        dense symmetrised chi0bar by the Adler-Wiser sum over states
                  at omega = 0 (Eq. AdlerWiser), its eigendecomposition
                  (Eq. eigendecompzerofreq), and the free-electron closed form.
* ``screening``   reducible chibar = (1 - chi0bar)^{-1} chi0bar, epsbar^{-1} and
                  W^p at omega = 0 (Eqs. linearalgebrachichi0, epsilonandchi,
                  Wpnondiag), dense and in the PDEP basis.
* ``lanczos``     Lanczos chains of the deflated Hamiltonian P_c H P_c and the
                  omega-independent poles and weights of M_c(omega) (Sec. II D,
                  Eqs. MCdef, MCfinal), and the exact sum over empty states.
* ``iterative``   the same Kohn-Sham states, Sternheimer solutions and chi0bar
                  phi without dense matrices (Lanczos eigensolver and
                  preconditioned block CG on the grid-applied H), for systems
                  whose dense H does not fit (the 64x64x192 interface).

Pins (tests/test_oracle_*.py): free-electron closed form, finite-difference
density and second-order band-energy response, brute-force matrix elements,
Sternheimer = sum over states, symmetry, negative semi-definiteness,
charge neutrality, invariance under V -> V + const.  The paper prints no
worked numerical example for this path, so no pin uses printed values.
"""
from . import basis, hamiltonian, response, pdep, screening, lanczos, iterative  # noqa: F401

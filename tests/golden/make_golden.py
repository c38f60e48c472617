"""Writes the stored expected values of tests/golden/ from the oracle alone.

free_electron_24cube_nocc7.txt: the 26 most negative eigenvalues of chi0bar
at omega = 0 for V = 0 on the 24^3 grid of a cubic cell of edge 10 bohr
(alias-free cutoff, 799 plane waves), 7 occupied states (the closed shell
k = 0 plus the six |k| = 2 pi / L waves).  With V = 0 the Kohn-Sham states
are plane waves and the Adler-Wiser sum at omega = 0 (Sec. II A, Eq.
AdlerWiser; symmetrised with v^{1/2} = sqrt(4 pi)/|G|, Eq. symmoperator) is
diagonal in G, so each eigenvalue is the closed form
    lambda(G) = 16 pi / (Omega |G|^2) sum_{k occ, k+G empty} 1/(eps_k - eps_{k+G}),
eps_k = |k|^2 / 2, k + G inside the basis sphere.  The 26 values end on a
complete multiplet (6 + 8 + 12).

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.basis import Basis  # noqa: E402
from oracle.pdep import free_electron_chi0bar  # noqa: E402

GRID = (24, 24, 24)
CELL = (10.0, 10.0, 10.0)
N_OCC = 7
N_KEEP = 26
NAME = "free_electron_24cube_nocc7.txt"


def values() -> np.ndarray:
    b = Basis(GRID, CELL)
    return np.sort(free_electron_chi0bar(b, N_OCC))[:N_KEEP]


def write(path: str) -> None:
    lam = values()
    with open(path, "w") as f:
        f.write("# Free-electron chi0bar eigenvalues at omega = 0 (V = 0), most negative first.\n")
        f.write("# Closed form of the Adler-Wiser sum (Sec. II A, Eq. AdlerWiser) symmetrised with\n")
        f.write("# sqrt(4 pi)/|G| (Eq. symmoperator); written by tests/golden/make_golden.py.\n")
        f.write(f"# grid {GRID[0]} {GRID[1]} {GRID[2]}  cell {CELL[0]} {CELL[1]} {CELL[2]} bohr"
                f"  n_occ {N_OCC}  n_pw 799  (Hartree units)\n")
        for i, x in enumerate(lam):
            f.write(f"{i} {x:.17e}\n")


def read(path: str) -> np.ndarray:
    return np.array([float(line.split()[1]) for line in open(path)
                     if line.strip() and not line.startswith("#")])


if __name__ == "__main__":
    write(os.path.join(HERE, NAME))

"""Stored expected values of tests/golden/ (written by make_golden.py from the
oracle's closed forms) against the oracle's general code paths.

free_electron_24cube_nocc7.txt: the dense Adler-Wiser chi0bar of the oracle
(pair densities by grid products, sum over all 792 empty states, dense
eigh; Sec. II A) for V = 0 on the 24^3 grid reproduces the stored
closed-form eigenvalues, and regenerating the file gives the stored values.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def _stored():
    return make_golden.read(os.path.join(HERE, "golden", make_golden.NAME))


def test_stored_file_is_current():
    lam = _stored()
    assert lam.shape == (make_golden.N_KEEP,)
    np.testing.assert_allclose(lam, make_golden.values(), rtol=1e-15, atol=0)


def test_dense_oracle_reproduces_free_electron_golden():
    from oracle.basis import Basis
    from oracle.hamiltonian import ks_states
    from oracle.pdep import chi0bar_dense
    b = Basis(make_golden.GRID, make_golden.CELL)
    assert b.n_pw == 799
    ks = ks_states(b, np.zeros(b.grid), make_golden.N_OCC)
    lam = np.linalg.eigvalsh(chi0bar_dense(b, ks))
    stored = _stored()
    np.testing.assert_allclose(lam[: make_golden.N_KEEP], stored, rtol=1e-12, atol=0)
    # the stored list ends on a complete multiplet
    assert lam[make_golden.N_KEEP] > stored[-1] + 1e-3

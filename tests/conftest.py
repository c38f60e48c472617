import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def tiny_system():
    import synthetic
    return synthetic.make_system("tiny")


@pytest.fixture(scope="session")
def tiny_oracle(tiny_system):
    """Basis, Kohn-Sham states and dense Hamiltonian of the 24^3 workload."""
    from oracle.basis import Basis
    from oracle.hamiltonian import dense_hamiltonian, ks_states
    b = Basis(tiny_system.grid, tiny_system.cell)
    ks = ks_states(b, tiny_system.v_r, tiny_system.n_occ)
    h = dense_hamiltonian(b, tiny_system.v_r)
    return b, ks, h


@pytest.fixture(scope="session")
def tiny_chib(tiny_oracle):
    from oracle.pdep import chi0bar_dense
    b, ks, _ = tiny_oracle
    return chi0bar_dense(b, ks)

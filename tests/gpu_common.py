"""Shared helpers of the GPU parity tests (not collected as a test module)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@functools.lru_cache(maxsize=None)
def lib_ready():
    from paper_1501_03141_gb300 import _abi, build
    build.build(bounds_check=_abi.BOUNDS_CHECK)
    return True


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) /
                 max(np.linalg.norm(np.asarray(b)), 1e-300))


@functools.lru_cache(maxsize=None)
def oracle_for(name):
    """(system, basis, ks) of a named workload, computed once per session."""
    import synthetic
    from oracle.basis import Basis
    from oracle.hamiltonian import ks_states
    s = synthetic.make_system(name)
    b = Basis(s.grid, s.cell)
    ks = ks_states(b, s.v_r, s.n_occ)
    return s, b, ks


def sign_align(psi_gpu, ks):
    """Per-state sign that maps the GPU's psi_v onto the oracle's."""
    n = psi_gpu.shape[0]
    ov = np.sum(psi_gpu * ks.C[:, :n].T, axis=1)
    assert np.all(np.abs(np.abs(ov) - 1.0) < 1e-8), ov
    return np.sign(ov)

"""chi0bar applied through Sternheimer solves (Eqs. stern, deltani,
chiisamatrixinpdep) against the oracle's dense Adler-Wiser chi0bar, and the
density response dn(r) against the oracle's.

Tolerances: 1e-8 relative on chi0bar phi and 1e-7 relative on dn (FP64
path); 1e-6 for the mixed path.
"""
import numpy as np
import pytest

import synthetic
from oracle import response
from oracle.pdep import chi0bar_dense

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_dense():
    s, b, ks = oracle_for("tiny")
    return chi0bar_dense(b, ks)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
@pytest.mark.parametrize("n_pert", [1, 4, 5])
def test_tiny_chi0(precision, tol, n_pert, tiny_dense):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    phi = synthetic.random_vectors(30 + n_pert, n_pert, b.n_pdep_dim)
    dn = np.empty((n_pert, b.n_r))
    with pg.Context(s, precision=precision) as ctx:
        out = ctx.chi0_apply(phi, dn=dn)
    assert rel(out, phi @ tiny_dense) < tol
    _, dn_ref = response.chi0bar_apply(b, ks, phi, return_dn=True)
    assert rel(dn, dn_ref.reshape(n_pert, -1)) < 10 * tol
    # no net charge in the response
    assert abs(dn.sum()) * b.omega / b.n_r < 1e-10 * np.abs(dn).sum() * b.omega / b.n_r


def test_tiny_chi0_device_buffers(tiny_dense):
    need_gpu()
    lib_ready()
    import torch
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    phi = torch.tensor(synthetic.random_vectors(40, 3, b.n_pdep_dim), device="cuda")
    with pg.Context(s) as ctx:
        out = ctx.chi0_apply(phi)
        torch.cuda.synchronize()
    assert out.is_cuda
    assert rel(out.cpu().numpy(), phi.cpu().numpy() @ tiny_dense) < 1e-8


def test_cube48_sampled():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("cube48")
    phi = synthetic.random_vectors(41, 4, b.n_pdep_dim)
    dn = np.empty((4, b.n_r))
    with pg.Context(s) as ctx:
        out = ctx.chi0_apply(phi, dn=dn)
    ref, dn_ref = response.chi0bar_apply(b, ks, phi, return_dn=True)
    assert rel(out, ref) < 1e-8
    assert rel(dn, dn_ref.reshape(4, -1)) < 1e-7

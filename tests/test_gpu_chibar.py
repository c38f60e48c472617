"""chibar with the Hartree-only self-consistent response (Sec. II C, Eqs. LF,
LFHartree, linearalgebrachichi0) through the C ABI.

* 24^3: against the oracle's dense Dyson solve (1 - chi0bar)^{-1} chi0bar,
  FP64 (1e-8) and mixed (1e-6); on an exact PDEP eigenvector chibar phi =
  lambda/(1 - lambda) phi;
* 48^3 (mixed): the Dyson identity chibar phi - chi0bar (chibar phi) =
  chi0bar phi with chi0bar applied through chi0_apply;
* argument errors, n = 0, and the iteration cap.
"""
import numpy as np
import pytest

import synthetic
from oracle import screening
from oracle.pdep import chi0bar_dense, pdep_reference

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_chib():
    s, b, ks = oracle_for("tiny")
    return chi0bar_dense(b, ks)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_tiny_against_dyson(precision, tol, tiny_chib):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    phi = synthetic.random_vectors(71, 4, b.n_pdep_dim)
    with pg.Context(s, precision=precision) as ctx:
        out, its = ctx.chibar_apply(phi, tol=1e-10)
    ref = phi @ screening.chibar_dyson(tiny_chib).T
    assert rel(out, ref) < tol
    assert 0 < its < 200


def test_tiny_eigenvector(tiny_chib):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, vec = pdep_reference(tiny_chib, 3)
    with pg.Context(s) as ctx:
        out, _ = ctx.chibar_apply(np.ascontiguousarray(vec.T), tol=1e-10)
    for i in range(3):
        assert rel(out[i], lam[i] / (1 - lam[i]) * vec[:, i]) < 1e-7


def test_cube48_dyson_identity():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s = synthetic.make_system("cube48")
    with pg.Context(s, precision=1) as ctx:
        phi = synthetic.random_vectors(72, 2, ctx.sizes()["n_pdep_dim"])
        chi, its = ctx.chibar_apply(phi, tol=1e-9)
        lhs = chi - ctx.chi0_apply(chi)
        rhs = ctx.chi0_apply(phi)
    assert rel(lhs, rhs) < 1e-7
    assert its > 0


def test_errors_and_cap():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    phi = synthetic.random_vectors(73, 2, b.n_pdep_dim)
    with pg.Context(s) as ctx:
        with pytest.raises(pg.PdepError):
            ctx.chibar_apply(phi, tol=0.0)
        with pytest.raises(pg.PdepError):
            ctx.chibar_apply(phi, max_iter=0)
        out, its = ctx.chibar_apply(np.empty((0, b.n_pdep_dim)))
        assert out.shape == (0, b.n_pdep_dim) and its == 0
        with pytest.raises(pg.PdepError) as e:
            ctx.chibar_apply(phi, tol=1e-14, max_iter=2)
        assert e.value.status == pg._abi.PDEP_ERR_NOT_CONVERGED

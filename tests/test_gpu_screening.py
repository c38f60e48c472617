"""Screening at omega = 0 from PDEP eigenpairs (Sec. II A) through the C ABI.

* The library's low-rank chibar, epsbar^{-1} and W^p applied to random
  vectors equal the oracle's PDEP form evaluated with the same eigenpairs
  (pure linear algebra: 1e-12), host and device buffers;
* with the GPU's own Davidson eigenpairs of the 24^3 workload they equal the
  oracle's PDEP form built from the dense chi0bar's exact eigenpairs (1e-6);
* at 48^3 the same identities hold on sampled vectors with random
  orthonormal stand-in eigenvectors and NSD eigenvalues;
* argument errors: unknown kind, lambda >= 1, n_pdep out of range; n = 0.
"""
import numpy as np
import pytest

from oracle import screening
from oracle.pdep import chi0bar_dense, pdep_reference

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu

KINDS = ("chibar", "epsinv", "wp")


def _orthonormal(rng, dim, k):
    q, _ = np.linalg.qr(rng.standard_normal((dim, k)))
    return q


@pytest.mark.parametrize("kind", KINDS)
def test_linear_algebra_parity_tiny(kind):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, _ = oracle_for("tiny")
    rng = np.random.default_rng(11)
    dim = b.n_pdep_dim
    vecs = _orthonormal(rng, dim, 16)
    lam = -np.sort(rng.uniform(0.05, 3.0, 16))[::-1]
    f = rng.standard_normal((5, dim))
    with pg.Context(s) as ctx:
        out = ctx.screening_apply(kind, lam, np.ascontiguousarray(vecs.T), f)
    ref = screening.pdep_screening(kind, lam, vecs, f, b.sqrt_coulomb())
    assert rel(out, ref) < 1e-12


def test_device_buffers_and_empty():
    need_gpu()
    lib_ready()
    import torch
    import paper_1501_03141_gb300 as pg
    s, b, _ = oracle_for("tiny")
    rng = np.random.default_rng(12)
    dim = b.n_pdep_dim
    vecs = _orthonormal(rng, dim, 9)
    lam = -rng.uniform(0.01, 2.0, 9)
    f = rng.standard_normal((3, dim))
    with pg.Context(s) as ctx:
        d = torch.device("cuda:0")
        out = ctx.screening_apply("wp", torch.tensor(lam, device=d),
                                  torch.tensor(np.ascontiguousarray(vecs.T), device=d),
                                  torch.tensor(f, device=d))
        empty = ctx.screening_apply("chibar", lam, np.ascontiguousarray(vecs.T),
                                    np.empty((0, dim)))
    ref = screening.pdep_screening("wp", lam, vecs, f, b.sqrt_coulomb())
    assert rel(out.cpu().numpy(), ref) < 1e-12
    assert empty.shape == (0, dim)


def test_with_davidson_eigenpairs_tiny():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam_x, vec_x = pdep_reference(chi0bar_dense(b, ks), s.n_pdep)
    rng = np.random.default_rng(13)
    f = rng.standard_normal((4, b.n_pdep_dim))
    with pg.Context(s) as ctx:
        ev, evec, st = ctx.pdep_solve()
        assert st["converged"] == 1
        evec = evec.reshape(s.n_pdep, b.n_pdep_dim)
        for kind in KINDS:
            out = ctx.screening_apply(kind, ev, evec, f)
            ref = screening.pdep_screening(kind, lam_x, vec_x, f, b.sqrt_coulomb())
            assert rel(out, ref) < 1e-6, kind


def test_sampled_cube48():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    import synthetic
    s = synthetic.make_system("cube48")
    with pg.Context(s) as ctx:
        dim = ctx.sizes()["n_pdep_dim"]
        from oracle.basis import Basis
        b = Basis(s.grid, s.cell)
        assert b.n_pdep_dim == dim
        rng = np.random.default_rng(14)
        vecs = _orthonormal(rng, dim, 128)
        lam = -np.sort(rng.uniform(0.01, 5.0, 128))[::-1]
        f = rng.standard_normal((7, dim))
        for kind in KINDS:
            out = ctx.screening_apply(kind, lam, np.ascontiguousarray(vecs.T), f)
            ref = screening.pdep_screening(kind, lam, vecs, f, b.sqrt_coulomb())
            assert rel(out, ref) < 1e-12, kind


def test_argument_errors():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, _ = oracle_for("tiny")
    dim = b.n_pdep_dim
    rng = np.random.default_rng(15)
    vecs = np.ascontiguousarray(_orthonormal(rng, dim, 4).T)
    f = rng.standard_normal((2, dim))
    with pg.Context(s) as ctx:
        with pytest.raises(pg.PdepError):
            ctx.screening_apply(3, -np.ones(4), vecs, f)
        with pytest.raises(pg.PdepError):
            ctx.screening_apply("chibar", np.array([-1.0, 0.5, 1.0, -2.0]), vecs, f)
        with pytest.raises(pg.PdepError):
            ctx.screening_apply("chibar", np.array([-1.0, np.nan, -1.0, -2.0]), vecs, f)
        with pytest.raises(pg.PdepError):
            ctx.screening_apply("epsinv", np.empty(0), vecs[:0], f)

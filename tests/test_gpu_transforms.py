"""Sphere <-> grid transforms and H*psi (the FFT and fused H*psi kernels)
against the oracle, on every supported grid shape, FP64 and FP32.

Sizes: each shape runs the pruned column/slab kernels over several x-planes,
several column tiles and a ragged item count (odd vector counts leave the
second field of the last packed pair empty).
"""
import numpy as np
import pytest

import synthetic
from oracle.basis import Basis
from oracle.hamiltonian import apply_hamiltonian_grid, ks_states

from gpu_common import lib_ready, need_gpu, rel

pytestmark = pytest.mark.gpu

SHAPES = [
    ((24, 24, 24), (10.0, 10.0, 10.0)),
    ((32, 32, 32), (13.3, 13.3, 13.3)),
    ((40, 40, 40), (16.7, 16.7, 16.7)),
    ((48, 48, 48), (20.0, 20.0, 20.0)),
    ((64, 64, 64), (26.7, 26.7, 26.7)),
    ((64, 64, 192), (20.0, 20.0, 60.0)),
]


def _system(grid, cell, n_occ=2, seed=1):
    rng = np.random.default_rng(seed)
    c, d, w = synthetic.gaussian_wells(rng, 4, cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(grid, cell, c, d, w)
    return synthetic.System(name="t", grid=grid, cell=cell, v_r=v, n_occ=n_occ, n_pdep=2, seed=seed)


@pytest.mark.parametrize("grid,cell", SHAPES)
def test_to_grid_and_hpsi(grid, cell):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s = _system(grid, cell)
    b = Basis(grid, cell)
    with pg.Context(s) as ctx:
        assert ctx.sizes() == {"n_pw": b.n_pw, "n_r": b.n_r, "n_pdep_dim": b.n_pw - 1}
        x = np.random.default_rng(2).standard_normal((3, b.n_pw))
        u = ctx.to_grid(x)
        assert rel(u.reshape(3, -1), b.coeffs_to_grid(x).reshape(3, -1)) < 1e-14
        ref = apply_hamiltonian_grid(b, s.v_r, x)
        assert rel(ctx.apply_hamiltonian(x), ref) < 1e-14
        assert rel(ctx.apply_hamiltonian(x, precision=pg.PDEP_MIXED), ref) < 2e-7
        # double-float transforms (the mixed refinement's A delta): ~48-bit arithmetic
        assert rel(ctx.apply_hamiltonian(x, precision=pg.PDEP_APPLY_DF64), ref) < 1e-13
        # single vector (odd item) and a per-vector check
        one = ctx.apply_hamiltonian(x[1:2].copy())
        assert rel(one[0], ref[1]) < 1e-14
    # FP32: the fused one-launch transform (cubic 24^3 .. 48^3) and the
    # three-launch form agree to FP32 rounding
    with pg.Context(s, fused_hpsi=0) as ctx:
        y3 = ctx.apply_hamiltonian(x, precision=pg.PDEP_MIXED)
    with pg.Context(s) as ctx:
        y1 = ctx.apply_hamiltonian(x, precision=pg.PDEP_MIXED)
    assert rel(y1, ref) < 2e-7 and rel(y3, ref) < 2e-7 and rel(y1, y3) < 2e-7


@pytest.mark.parametrize("grid,cell", SHAPES[:4])
def test_setup_eigenpairs(grid, cell):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s = _system(grid, cell, n_occ=3, seed=4)
    b = Basis(grid, cell)
    ks = ks_states(b, s.v_r, 3)
    # eigenpairs only: accept whatever gap this draw has
    with pg.Context(s, gap_min=1e-9) as ctx:
        psi, eps = ctx.occupied()
    np.testing.assert_allclose(eps, ks.eps[:4], atol=1e-10)
    ov = np.abs(np.sum(psi * ks.C[:, :3].T, axis=1))
    np.testing.assert_allclose(ov, 1.0, atol=1e-9)


def test_empty_batch_is_noop():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s = synthetic.make_system("tiny")
    with pg.Context(s) as ctx:
        x = np.zeros((0, ctx.sizes()["n_pw"]))
        assert ctx.apply_hamiltonian(x).shape == (0, ctx.sizes()["n_pw"])

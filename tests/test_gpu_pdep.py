"""Davidson PDEP solve (Sec. II C) through the C ABI.

24^3 workload: the 16 most negative eigenvalues against the oracle's dense
chi0bar eigendecomposition (1e-8 relative, FP64; 1e-6 mixed), and the
eigenvector subspace against the oracle's (projector distance).
48^3 workload at the bench configuration (6 Davidson iterations): the
mixed path against the FP64 path eigenvalue by eigenvalue (1e-6), and
the oracle's chi0bar applied to sampled GPU eigenvectors reproduces the
Rayleigh quotients, with Cauchy interlacing against nothing smaller than
the dense-free bound lambda_i >= ... checked through residual norms.
"""
import numpy as np
import pytest

from oracle import response
from oracle.pdep import chi0bar_dense, pdep_reference

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_ref():
    s, b, ks = oracle_for("tiny")
    return pdep_reference(chi0bar_dense(b, ks), s.n_pdep)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6), (2, 1e-6)])
def test_tiny_eigenpairs(precision, tol, tiny_ref):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, vec = tiny_ref
    with pg.Context(s, precision=precision) as ctx:
        ev, evec, st = ctx.pdep_solve()
    assert st["converged"] == 1
    err = np.abs(ev - lam) / np.abs(lam)
    assert err.max() < tol, err
    V = evec.reshape(s.n_pdep, b.n_pdep_dim).T
    # same invariant subspace (no degeneracy at the cut: checked below)
    assert (lam[-1] - ev[-1]) == pytest.approx(0.0, abs=1e-6 * abs(lam[-1]))
    P1 = V @ V.T
    P2 = vec @ vec.T
    assert np.linalg.norm(P1 - P2) < 1e-5
    np.testing.assert_allclose(V.T @ V, np.eye(s.n_pdep), atol=1e-10)


def test_tiny_user_start_block(tiny_ref):
    need_gpu()
    lib_ready()
    import synthetic
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, _ = tiny_ref
    phi0 = synthetic.random_vectors(5, s.n_pdep, b.n_pdep_dim)
    with pg.Context(s) as ctx:
        ev, _, _ = ctx.pdep_solve(phi0=phi0)
    assert (np.abs(ev - lam) / np.abs(lam)).max() < 1e-8


def test_cube48_mixed_vs_fp64_and_rayleigh():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("cube48")
    opts = dict(dav_tol=0.0, dav_max_iter=6)
    with pg.Context(s, precision=pg.PDEP_FP64, **opts) as ctx:
        ev64, vec64, st64 = ctx.pdep_solve()
    with pg.Context(s, precision=pg.PDEP_MIXED, **opts) as ctx:
        ev32, vec32, st32 = ctx.pdep_solve()
    with pg.Context(s, precision=pg.PDEP_MIXED_BF16, **opts) as ctx:
        ev16, _, st16 = ctx.pdep_solve()
    assert st64["dav_iterations"] == 6 and st32["dav_iterations"] == 6
    assert st16["dav_iterations"] == 6 and st16["proj_variant"] == 3
    assert st16["max_cg_residual"] <= 1e-10
    err = np.abs(ev32 - ev64) / np.abs(ev64)
    assert err.max() < 1e-6, err
    err16 = np.abs(ev16 - ev64) / np.abs(ev64)
    print(f"cube48, 128 eigenvalues vs FP64: TF32 mode {err.max():.2e}, BF16 mode {err16.max():.2e}")
    assert err16.max() < 1e-6, err16
    assert np.all(np.diff(ev64) >= 0) and ev64[-1] < 0
    # oracle chi0bar on sampled eigenvectors: Rayleigh quotients equal the Ritz values
    V = vec64.reshape(s.n_pdep, b.n_pdep_dim)
    pick = [0, 1, 63, 127]
    cv = response.chi0bar_apply(b, ks, V[pick])
    rq = np.sum(cv * V[pick], axis=1)
    np.testing.assert_allclose(rq, ev64[pick], rtol=1e-8)


def test_ritz_interlacing_and_monotone(tiny_ref):
    """After k Davidson iterations (no restart yet) the Ritz values interlace:
    theta_i >= lambda_i (Cauchy), and growing the subspace lowers each one."""
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, _ = tiny_ref
    thetas = []
    for k in (1, 2, 3):
        with pg.Context(s, dav_tol=0.0, dav_max_iter=k) as ctx:
            ev, _, st = ctx.pdep_solve(allow_unconverged=True)
        assert st["dav_iterations"] == k
        thetas.append(ev)
    tol = 1e-10 * abs(lam[0])
    for th in thetas:
        assert np.all(th >= lam - tol), th - lam
    assert np.all(thetas[1] <= thetas[0] + tol)
    assert np.all(thetas[2] <= thetas[1] + tol)


def test_checkpoint_resume(tiny_ref, tmp_path):
    """A run cut after two Davidson iterations is saved to disk; resuming from
    the saved vectors converges to the same eigenpairs in fewer iterations
    than a cold start."""
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, _ = tiny_ref
    with pg.Context(s, dav_tol=0.0, dav_max_iter=2) as ctx:
        _, evec, _ = ctx.pdep_solve(allow_unconverged=True)
    ck = tmp_path / "pdep_vectors.npy"
    np.save(ck, evec.reshape(s.n_pdep, b.n_pdep_dim))
    with pg.Context(s) as ctx:
        ev_cold, _, st_cold = ctx.pdep_solve()
        ev_warm, _, st_warm = ctx.pdep_solve(phi0=np.load(ck))
    assert st_cold["converged"] == 1 and st_warm["converged"] == 1
    assert (np.abs(ev_warm - lam) / np.abs(lam)).max() < 1e-8
    assert (np.abs(ev_warm - ev_cold) / np.abs(lam)).max() < 1e-8
    assert st_warm["dav_iterations"] < st_cold["dav_iterations"]


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_free_electron_golden(precision, tol):
    """V = 0 on the 24^3 grid, 7 occupied states: the GPU's PDEP eigenvalues
    against the stored closed-form values (tests/golden), through the first
    two complete multiplets (6 + 8); the occupied shell and the Sternheimer
    operators are degenerate."""
    need_gpu()
    lib_ready()
    import os
    import sys
    import synthetic
    import paper_1501_03141_gb300 as pg
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden
    stored = make_golden.read(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                           make_golden.NAME))
    s = synthetic.System(name="free24", grid=make_golden.GRID, cell=make_golden.CELL,
                         v_r=np.zeros(make_golden.GRID), n_occ=make_golden.N_OCC, n_pdep=14,
                         seed=0)
    with pg.Context(s, precision=precision) as ctx:
        assert ctx.sizes()["n_pw"] == 799
        ev, _, st = ctx.pdep_solve()
    assert st["converged"] == 1
    err = np.abs(ev - stored[:14]) / np.abs(stored[:14])
    assert err.max() < tol, err

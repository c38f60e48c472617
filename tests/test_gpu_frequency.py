"""Body of chi0bar at imaginary frequencies from Lanczos chains (Sec. II B,
Eq. finalB; Sec. II D) and Lambda = (1 - B)^{-1} B, through the C ABI.

* 24^3, 64-step chains, the oracle's exact PDEP eigenvectors: B(i nu) against
  phi^T chi0bar(i nu) phi from the oracle's dense Adler-Wiser sum at nu = 0,
  0.5, 2 (1e-9), B(0) = diag(lambda) (1e-9), Lambda against (1 - B)^{-1} B
  of the oracle's B (1e-9);
* 24^3, 40-step chains: against the same Lanczos construction done by the
  oracle (1e-9, the truncation error is shared);
* 48^3 with the GPU's own Davidson eigenvectors (6 iterations): B symmetric,
  negative definite, decreasing in magnitude with nu, B(0) close to
  diag(theta) of the Rayleigh-Ritz values;
* argument errors.
"""
import numpy as np
import pytest

from oracle import lanczos as lz, response, screening
from oracle.pdep import chi0bar_dense, pdep_reference

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_pdep():
    s, b, ks = oracle_for("tiny")
    return pdep_reference(chi0bar_dense(b, ks), s.n_pdep)


def test_tiny_against_dense(tiny_pdep):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    lam, vec = tiny_pdep
    nus = np.array([0.0, 0.5, 2.0])
    with pg.Context(s) as ctx:
        B, L = ctx.chi0_imag(np.ascontiguousarray(vec.T), nus, n_steps=64)
    for f, nu in enumerate(nus):
        Bx = screening.pdep_body(chi0bar_dense(b, ks, nu=nu), vec)
        assert rel(B[f], Bx) < 1e-9, nu
        assert rel(L[f], screening.lambda_body(Bx)) < 1e-9, nu
    assert rel(np.diag(B[0]), lam) < 1e-9


def test_tiny_against_oracle_lanczos(tiny_pdep):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    from oracle.hamiltonian import dense_hamiltonian
    s, b, ks = oracle_for("tiny")
    lam, vec = tiny_pdep
    K, nu = 40, 0.3
    hd = lz.deflated_hamiltonian(dense_hamiltonian(b, s.v_r), ks)
    u = response.occupied_grid(b, ks)
    vh = b.sqrt_coulomb()
    V = ks.C[:, : s.n_occ]
    R = np.zeros((s.n_pdep, s.n_occ, b.n_pw))
    for j in range(s.n_pdep):
        dv = b.coeffs_to_grid(np.concatenate([vh * vec[:, j], [0.0]])) / np.sqrt(b.omega)
        w = response.perturbation_projections(b, u, dv)
        R[j] = w - (w @ V) @ V.T
    Bo = np.zeros((s.n_pdep, s.n_pdep))
    for v in range(s.n_occ):
        for j in range(s.n_pdep):
            a, bb, Q = lz.lanczos_chain(hd, R[j, v], K)
            d, wgt = lz.lanczos_poles_weights(a, bb, Q, R[:, v])
            D = ks.eps[v] - d
            Bo[:, j] += 4.0 * (wgt @ (D / (D * D + nu * nu)))
    Bo = 0.5 * (Bo + Bo.T)
    with pg.Context(s) as ctx:
        B, _ = ctx.chi0_imag(np.ascontiguousarray(vec.T), [nu], n_steps=K, with_lambda=False)
    assert rel(B[0], Bo) < 1e-9


def test_cube48_properties():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    import synthetic
    s = synthetic.make_system("cube48")
    with pg.Context(s, precision=1, dav_tol=0.0, dav_max_iter=6) as ctx:
        th, evec, _ = ctx.pdep_solve()
        phi = evec.reshape(s.n_pdep, -1)[:32]
        B, L = ctx.chi0_imag(np.ascontiguousarray(phi), [0.0, 0.5, 2.0], n_steps=40)
    for f in range(3):
        assert np.abs(B[f] - B[f].T).max() == 0.0
        assert np.linalg.eigvalsh(B[f]).max() < 0.0
    assert np.abs(np.linalg.eigvalsh(B[2])).max() < np.abs(np.linalg.eigvalsh(B[1])).max()
    assert np.abs(np.linalg.eigvalsh(B[1])).max() < np.abs(np.linalg.eigvalsh(B[0])).max()
    # at nu = 0 the chains resolve eps_v next to a 3 mHa gap: loose
    assert rel(np.diag(B[0]), th[:32]) < 1e-2
    mu = np.linalg.eigvalsh(B[1])
    assert rel(np.sort(np.linalg.eigvalsh(L[1])), np.sort(mu / (1 - mu))) < 1e-10


def test_argument_errors(tiny_pdep):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    _, vec = tiny_pdep
    phi = np.ascontiguousarray(vec.T)
    with pg.Context(s) as ctx:
        with pytest.raises(pg.PdepError):
            ctx.chi0_imag(phi, [1.0], n_steps=65)
        with pytest.raises(pg.PdepError):
            ctx.chi0_imag(phi, [np.nan], n_steps=8)
        B, L = ctx.chi0_imag(phi, np.empty(0), n_steps=8)
        assert B.shape == (0, s.n_pdep, s.n_pdep)

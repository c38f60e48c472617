"""Lanczos chains of the deflated Hamiltonian (Sec. II D) through the C ABI.

* 24^3: the recursion coefficients of 16-step chains against the oracle's
  (1e-10 on alpha, beta); the poles (1e-10) and M_c(omega) from the poles and
  weights (1e-10) for 40-step chains against the oracle's chains;
* 64-step chains approach the exact sum over empty states as closely as the
  oracle's 64-step chains do (1e-5 here), at imaginary and complex frequencies;
* 48^3 (the bench system): 40-step chains on two start vectors against the
  oracle's chains with the dense Hamiltonian (M_c to 1e-9);
* a start vector inside the occupied space gives an empty chain; argument
  errors; device buffers.
"""
import numpy as np
import pytest

import synthetic
from oracle import lanczos as lz
from oracle.hamiltonian import dense_hamiltonian

from gpu_common import lib_ready, need_gpu, oracle_for, rel

pytestmark = pytest.mark.gpu

OMEGAS = np.array([0.3j, 1j, 4j, 20j, -2.0 + 0.5j, 1.5 + 2j])


def _oracle_chains(s, b, ks, h, R, L, K):
    hd = lz.deflated_hamiltonian(h, ks)
    v = ks.C[:, : ks.n_occ]
    pcf = lambda x: x - v @ (v.T @ x)
    out = []
    for r in R:
        a, bb, Q = lz.lanczos_chain(hd, r, K, pc=pcf)
        d, w = lz.lanczos_poles_weights(a, bb, Q, L)
        out.append((a, bb, d, w))
    return out


@pytest.fixture(scope="module")
def tiny_h():
    s, b, ks = oracle_for("tiny")
    return dense_hamiltonian(b, s.v_r)


@pytest.mark.parametrize("K", [16, 40])
def test_tiny_against_oracle_chains(K, tiny_h):
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    rng = np.random.default_rng(40 + K)
    R = rng.standard_normal((5, b.n_pw))
    L = rng.standard_normal((3, b.n_pw))
    with pg.Context(s) as ctx:
        poles, weights, alpha, beta = ctx.lanczos(R, K, L)
    ref = _oracle_chains(s, b, ks, tiny_h, R, L, K)
    for j, (a, bb, d, w) in enumerate(ref):
        m_ref = lz.lanczos_resolvent(d, w, OMEGAS)
        m = lz.lanczos_resolvent(poles[j], weights[j], OMEGAS)
        assert rel(m, m_ref) < 1e-10
        if K == 16:
            assert rel(alpha[j], a) < 1e-10 and rel(beta[j], bb) < 1e-10
            assert rel(poles[j], d) < 1e-10


def test_tiny_converges_to_sum_over_states(tiny_h):
    """64-step chains: as close to the exact sum over empty states as the
    oracle's own 64-step chains (the truncation error of Eq. MCfinal)."""
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    rng = np.random.default_rng(7)
    R = rng.standard_normal((2, b.n_pw))
    L = rng.standard_normal((2, b.n_pw))
    with pg.Context(s) as ctx:
        poles, weights, _, _ = ctx.lanczos(R, 64, L)
    ref = _oracle_chains(s, b, ks, tiny_h, R, L, 64)
    for j in range(2):
        ex = lz.resolvent_sos(ks, L, R[j], OMEGAS)
        m = lz.lanczos_resolvent(poles[j], weights[j], OMEGAS)
        m_or = lz.lanczos_resolvent(ref[j][2], ref[j][3], OMEGAS)
        assert rel(m, ex) < 1e-5
        assert rel(m, ex) < 1.5 * rel(m_or, ex) + 1e-10
        assert rel(m, m_or) < 1e-7


def test_cube48_against_oracle():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("cube48")
    h = dense_hamiltonian(b, s.v_r)
    rng = np.random.default_rng(9)
    R = rng.standard_normal((2, b.n_pw))
    L = rng.standard_normal((2, b.n_pw))
    with pg.Context(s) as ctx:
        poles, weights, alpha, _ = ctx.lanczos(R, 40, L)
    ref = _oracle_chains(s, b, ks, h, R, L, 40)
    for j, (a, bb, d, w) in enumerate(ref):
        assert rel(alpha[j][:10], a[:10]) < 1e-10
        m = lz.lanczos_resolvent(poles[j], weights[j], OMEGAS)
        assert rel(m, lz.lanczos_resolvent(d, w, OMEGAS)) < 1e-9


def test_occupied_start_and_device_buffers():
    need_gpu()
    lib_ready()
    import torch
    import paper_1501_03141_gb300 as pg
    s, b, ks = oracle_for("tiny")
    with pg.Context(s) as ctx:
        psi, _ = ctx.occupied()
        R = np.stack([psi[0], np.random.default_rng(1).standard_normal(b.n_pw)])
        L = np.random.default_rng(2).standard_normal((1, b.n_pw))
        poles, weights, alpha, beta = ctx.lanczos(R, 8, L)
        assert beta[0, 0] < 1e-12 and np.abs(weights[0]).max() == 0.0
        assert beta[1, 0] > 1.0
        d = torch.device("cuda:0")
        Rd = torch.tensor(R, device=d)
        Ld = torch.tensor(L, device=d)
        pd = torch.empty((2, 8), dtype=torch.float64, device=d)
        wd = torch.empty((2, 1, 8), dtype=torch.float64, device=d)
        lib = ctx._lib
        from paper_1501_03141_gb300 import _abi
        _abi.check(lib.pdep_lanczos(ctx._h, 0, _abi.ptr(Rd), 2, 8, _abi.ptr(Ld), 1, _abi.ptr(pd),
                                    _abi.ptr(wd), None, None, None), "pdep_lanczos")
        assert np.allclose(pd.cpu().numpy(), poles, rtol=0, atol=1e-12)
        assert np.allclose(wd.cpu().numpy(), weights, rtol=0, atol=1e-12)
        with pytest.raises(pg.PdepError):
            ctx.lanczos(R, 65, L)
        with pytest.raises(pg.PdepError):
            ctx.lanczos(R, 0, L)

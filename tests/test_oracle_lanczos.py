"""Pins of the oracle's Lanczos chains of the deflated Hamiltonian (Sec. II D).

* moments: for a K-step chain started on R, <R^|H~^k|R^> = (T^k)_11 for every
  k < 2K (the defining property of the Lanczos tridiagonalisation), with the
  moments taken by repeated dense products, independent of the recursion;
* a K-step chain's Q is orthonormal and spans the Krylov space (checked for a
  short chain);
* Eq. MCfinal converges to the exact M_c(omega) = -sum_c <L|c><c|R>/(eps_c -
  omega) of the empty states as K grows, and matches it to 1e-10 once K
  covers the resolvent (imaginary and complex frequencies);
* the weights do not depend on omega and M_c is linear in L and in R;
* a planted mistake (the beta_n q_{n-1} term dropped) fails the moments pin.
"""
import numpy as np
import pytest

from oracle import lanczos as lz


@pytest.fixture(scope="module")
def tiny_lz(tiny_oracle, tiny_system):
    b, ks, h = tiny_oracle
    hd = lz.deflated_hamiltonian(h, ks)
    v = ks.C[:, : ks.n_occ]
    pcf = lambda x: x - v @ (v.T @ x)
    rng = np.random.default_rng(3)
    return b, ks, hd, pcf, rng.standard_normal(b.n_pw), rng.standard_normal((3, b.n_pw))


def _moments_error(hd, pcf, R, alpha, beta, K):
    T = lz.tridiagonal(alpha, beta)
    r1 = pcf(R) / np.linalg.norm(pcf(R))
    v = r1.copy()
    tk = np.eye(K)
    worst = 0.0
    for _ in range(2 * K):
        mom = r1 @ v
        worst = max(worst, abs(mom - tk[0, 0]) / max(abs(mom), 1e-300))
        v = hd @ v
        tk = tk @ T
    return worst


@pytest.mark.parametrize("K", [4, 8])
def test_moments(K, tiny_lz):
    b, ks, hd, pcf, R, L = tiny_lz
    a, bb, Q = lz.lanczos_chain(hd, R, K, pc=pcf)
    assert _moments_error(hd, pcf, R, a, bb, K) < 1e-12


def test_short_chain_orthonormal_krylov(tiny_lz):
    b, ks, hd, pcf, R, L = tiny_lz
    K = 10
    a, bb, Q = lz.lanczos_chain(hd, R, K, pc=pcf)
    np.testing.assert_allclose(Q @ Q.T, np.eye(K), atol=1e-12)
    # the chain stays in range(P_c) and spans the Krylov space of P_c R
    occ = ks.C[:, : ks.n_occ]
    assert np.abs(occ.T @ Q.T).max() < 1e-12
    kry = [pcf(R)]
    for _ in range(K - 1):
        kry.append(hd @ kry[-1])
    kq, _ = np.linalg.qr(np.array(kry).T)
    assert np.linalg.norm(Q.T - kq @ (kq.T @ Q.T)) < 1e-8
    assert bb[0] == pytest.approx(np.linalg.norm(pcf(R)), rel=1e-14)


def test_converges_to_sum_over_states(tiny_lz):
    b, ks, hd, pcf, R, L = tiny_lz
    om = np.array([0.5j, 1j, 3j, 10j, -2.0 + 1j])
    ex = lz.resolvent_sos(ks, L, R, om)
    errs = []
    for K in (10, 20, 40, 80):
        a, bb, Q = lz.lanczos_chain(hd, R, K, pc=pcf)
        d, w = lz.lanczos_poles_weights(a, bb, Q, L)
        errs.append(np.abs(lz.lanczos_resolvent(d, w, om) - ex).max() / np.abs(ex).max())
    assert errs[-1] < 1e-10
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_linear_in_L_and_R(tiny_lz):
    b, ks, hd, pcf, R, L = tiny_lz
    K = 12
    om = np.array([1j, 2j])
    a, bb, Q = lz.lanczos_chain(hd, R, K, pc=pcf)
    d, w = lz.lanczos_poles_weights(a, bb, Q, L)
    m = lz.lanczos_resolvent(d, w, om)
    d2, w2 = lz.lanczos_poles_weights(a, bb, Q, L[0] + 2.0 * L[1])
    np.testing.assert_allclose(lz.lanczos_resolvent(d2, w2, om)[0], m[0] + 2.0 * m[1], rtol=1e-12)
    a3, b3, Q3 = lz.lanczos_chain(hd, -3.0 * R, K, pc=pcf)
    d3, w3 = lz.lanczos_poles_weights(a3, b3, Q3, L)
    np.testing.assert_allclose(lz.lanczos_resolvent(d3, w3, om), -3.0 * m, rtol=1e-11)


def test_planted_three_term_mistake_is_caught(tiny_lz):
    b, ks, hd, pcf, R, L = tiny_lz
    K = 6
    q0 = pcf(R)
    b0 = np.linalg.norm(q0)
    alpha, beta = np.zeros(K), np.zeros(K)
    beta[0] = b0
    q = q0 / b0
    for n in range(K):               # recursion without the beta_n q_{n-1} term
        w = hd @ q
        alpha[n] = q @ w
        w = w - alpha[n] * q
        if n + 1 < K:
            beta[n + 1] = np.linalg.norm(w)
            q = w / beta[n + 1]
    assert _moments_error(hd, pcf, R, alpha, beta, K) > 1e-6

"""Pins of the oracle's Sternheimer solution and density response (Sec. II C).

* Sternheimer by sum over empty states = Sternheimer by CG (Eq. stern);
* the SOS solution satisfies Eq. stern itself;
* finite differences of the ground-state density, n(r) = 2 sum_v |psi_v|^2,
  under H + eta dV reproduce dn of Eq. deltani (factor 4, sign, spin);
* the second derivative of the band energy E = 2 sum_v eps_v equals the
  quadratic form <dV|dn>, independent of the response code;
* the response carries no net charge.
"""
import numpy as np

import synthetic
from oracle.hamiltonian import ks_states
from oracle import response


def _dv(tiny_system, n=2, seed=77):
    return synthetic.random_grid_potentials(seed, n, tiny_system.grid, tiny_system.cell)


def test_sos_equals_cg(tiny_oracle, tiny_system):
    b, ks, h = tiny_oracle
    dv = _dv(tiny_system, 1)[0]
    sos = response.sternheimer_sos(b, ks, dv)
    cg, its, res = response.sternheimer_cg(b, ks, h, dv, tol=1e-12)
    assert np.all(res < 1e-11)
    np.testing.assert_allclose(cg, sos, atol=1e-9 * np.abs(sos).max())


def test_sos_solves_sternheimer(tiny_oracle, tiny_system):
    b, ks, h = tiny_oracle
    dv = _dv(tiny_system, 1, seed=78)[0]
    dpsi = response.sternheimer_sos(b, ks, dv)
    u = response.occupied_grid(b, ks)
    w = response.perturbation_projections(b, u, dv)
    Co = ks.C[:, : ks.n_occ]
    for v in range(ks.n_occ):
        lhs = h @ dpsi[v] - ks.eps[v] * dpsi[v]
        rhs = -(w[v] - Co @ (Co.T @ w[v]))
        assert np.linalg.norm(lhs - rhs) < 1e-10 * np.linalg.norm(rhs)
        assert np.abs(Co.T @ dpsi[v]).max() < 1e-12 * max(1.0, np.abs(dpsi[v]).max())


def test_density_finite_difference(tiny_oracle, tiny_system):
    b, ks, _ = tiny_oracle
    dv = _dv(tiny_system, 1, seed=79)[0]
    # the 14 mHa gap makes the response strongly nonlinear: error ~ (eta/gap)^2
    eta = 2e-5
    n_p = response.density_from_states(b, ks_states(b, tiny_system.v_r + eta * dv, ks.n_occ))
    n_m = response.density_from_states(b, ks_states(b, tiny_system.v_r - eta * dv, ks.n_occ))
    fd = (n_p - n_m) / (2 * eta)
    dn = response.density_response(b, response.occupied_grid(b, ks),
                                   response.sternheimer_sos(b, ks, dv))
    err = np.linalg.norm(fd - dn) / np.linalg.norm(dn)
    assert err < 2e-7, err


def test_band_energy_second_derivative(tiny_oracle, tiny_system):
    b, ks, _ = tiny_oracle
    dv = _dv(tiny_system, 1, seed=80)[0]
    eta = 2e-3
    e = [2.0 * np.sum(ks_states(b, tiny_system.v_r + s * eta * dv, ks.n_occ).eps[: ks.n_occ])
         for s in (-1, 0, 1)]
    d2 = (e[0] - 2 * e[1] + e[2]) / eta ** 2
    dn = response.density_response(b, response.occupied_grid(b, ks),
                                   response.sternheimer_sos(b, ks, dv))
    quad = np.sum(dv * dn) * b.omega / b.n_r
    assert quad < 0.0
    assert abs(d2 - quad) < 1e-4 * abs(quad), (d2, quad)


def test_charge_neutrality(tiny_oracle, tiny_system):
    b, ks, _ = tiny_oracle
    u = response.occupied_grid(b, ks)
    for dv in _dv(tiny_system, 2, seed=81):
        dn = response.density_response(b, u, response.sternheimer_sos(b, ks, dv, u))
        total = np.sum(dn) * b.omega / b.n_r
        assert abs(total) < 1e-12 * np.sum(np.abs(dn)) * b.omega / b.n_r

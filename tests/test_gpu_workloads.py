"""The other workloads of the hot path, through the C ABI.

Uneven batch (32 seeded systems, N in {24..64}, N_occ ~ U{8..96},
N_pdep = 2 N_occ): a context holding several members of different grid and
basis sizes is solved with pdep_solve(sys = -1); each member's eigenvalues
are compared with the oracle's dense chi0bar (1e-8 relative).

Interface (64x64x192 grid, 49 095 plane waves, 512 occupied states): too
large for the dense oracle, so properties that hold at any size are checked
on a sample of perturbations: the projected chi0bar is symmetric and
negative definite, the density response carries no charge, the mixed and
FP64 paths agree, every Sternheimer residual meets 1e-10, and the occupied
states satisfy H psi = eps psi under the oracle's own H application.
"""
import numpy as np
import pytest

import synthetic
from oracle.basis import Basis
from oracle.hamiltonian import apply_hamiltonian_grid, ks_states
from oracle.pdep import chi0bar_dense, pdep_reference

from gpu_common import lib_ready, need_gpu, rel

pytestmark = pytest.mark.gpu


def test_uneven_batch_members():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    batch = synthetic.make_batch()
    members = [batch[k] for k in (17, 8, 29)]          # 24^3, 32^3, 24^3; N_occ 16, 26, 14
    refs = []
    for s in members:
        b = Basis(s.grid, s.cell)
        ks = ks_states(b, s.v_r, s.n_occ)
        refs.append(pdep_reference(chi0bar_dense(b, ks), s.n_pdep)[0])
    with pg.Context(members, dav_tol=1e-8, dav_max_iter=40) as ctx:
        ev, _, st = ctx.pdep_solve(sys=-1)
    assert st["converged"] == 1
    off = 0
    for s, lam in zip(members, refs):
        got = ev[off:off + s.n_pdep]
        off += s.n_pdep
        err = np.abs(got - lam) / np.abs(lam)
        assert err.max() < 1e-8, (s.name, err.max())


@pytest.fixture(scope="module")
def interface():
    need_gpu()
    lib_ready()
    return synthetic.make_system("interface")


def test_interface_properties(interface):
    import paper_1501_03141_gb300 as pg
    s = interface
    b = Basis(s.grid, s.cell)
    n = 4
    phi = synthetic.random_vectors(61, n, b.n_pdep_dim)
    phi /= np.linalg.norm(phi, axis=1)[:, None]
    out = {}
    for prec in (pg.PDEP_FP64, pg.PDEP_MIXED):
        with pg.Context(s, precision=prec) as ctx:
            assert ctx.sizes()["n_pw"] == b.n_pw == 49095
            if prec == pg.PDEP_FP64:
                psi, eps = ctx.occupied()
                assert np.all(np.diff(eps) >= -1e-12) and eps[-1] - eps[-2] >= 1e-3
                pick = [0, 255, 511]
                hpsi = apply_hamiltonian_grid(b, s.v_r, psi[pick])
                res = np.linalg.norm(hpsi - eps[pick][:, None] * psi[pick], axis=1)
                assert res.max() < 1e-9, res
                dv = synthetic.random_grid_potentials(62, 1, s.grid, s.cell).reshape(1, -1)
                _, its, resid = ctx.sternheimer_solve(dv)
                assert resid.max() <= 1e-10 and its.min() > 0
            dn = np.empty((n, b.n_r))
            out[prec] = (ctx.chi0_apply(phi, dn=dn), dn)
    w, dn = out[pg.PDEP_FP64]
    M = phi @ w.T
    assert np.abs(M - M.T).max() < 1e-8 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).max() < 0
    assert np.abs(dn.sum(axis=1)).max() * b.omega / b.n_r < 1e-9 * np.abs(dn).sum() * b.omega / b.n_r
    assert rel(out[pg.PDEP_MIXED][0], w) < 1e-6

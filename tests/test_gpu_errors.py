"""Error paths of the C ABI (no GPU fault is ever provoked: every condition
is detected on the host or by a finite device loop)."""
import numpy as np
import pytest

import synthetic

from gpu_common import lib_ready, need_gpu

pytestmark = pytest.mark.gpu


def _pg():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    return pg


def test_unsupported_grid():
    pg = _pg()
    s = synthetic.System(name="x", grid=(20, 20, 20), cell=(8.0,) * 3, v_r=np.zeros((20,) * 3),
                         n_occ=1, n_pdep=1, seed=0)
    with pytest.raises(pg.PdepError) as e:
        pg.Context(s)
    assert e.value.status == 1


def test_no_gap():
    pg = _pg()
    # free electrons with 2 of the 6 degenerate |n| = 1 states occupied
    s = synthetic.System(name="x", grid=(24,) * 3, cell=(10.0,) * 3, v_r=np.zeros((24,) * 3),
                         n_occ=2, n_pdep=1, seed=0)
    with pytest.raises(pg.PdepError) as e:
        pg.Context(s)
    assert e.value.status == 4


def test_nonfinite_potential():
    pg = _pg()
    s = synthetic.make_system("tiny")
    v = s.v_r.copy()
    v[1, 2, 3] = np.nan
    bad = synthetic.System(name="x", grid=s.grid, cell=s.cell, v_r=v, n_occ=8, n_pdep=4, seed=0)
    with pytest.raises(pg.PdepError) as e:
        pg.Context(bad)
    assert e.value.status == 6


def test_iteration_cap_reports_not_converged():
    pg = _pg()
    s = synthetic.make_system("tiny")
    with pg.Context(s, cg_max_iter=3) as ctx:
        dv = synthetic.random_grid_potentials(3, 1, s.grid, s.cell).reshape(1, -1)
        with pytest.raises(pg.PdepError) as e:
            ctx.sternheimer_solve(dv)
        assert e.value.status == 5
        dpsi, its, res = ctx.sternheimer_solve(dv, allow_unconverged=True)
        # the cap holds for each refinement round
        assert its.max() <= 3 * ctx.options.max_refine and res.max() > 1e-10


def test_workspace_limit():
    pg = _pg()
    s = synthetic.make_system("tiny")
    with pytest.raises(pg.PdepError) as e:
        pg.Context(s, workspace_limit_bytes=1 << 16)
    assert e.value.status == 3


def test_bad_system_index():
    pg = _pg()
    s = synthetic.make_system("tiny")
    with pg.Context(s) as ctx:
        with pytest.raises(pg.PdepError):
            ctx.sizes(3)

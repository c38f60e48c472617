"""The device-driven Sternheimer loop and the enqueue-only boundary.

* Perturbation chunks (a workspace limit that splits one chi0bar
  application): chunked and unchunked results agree, and with a CG cap every
  chunk's output is still written.
* The CG loop captured as a CUDA graph (while node driven by a device control
  kernel) reproduces the host-driven loop: the same kernels in the same
  order, so the results agree to rounding (atomics in the split-K GEMMs and
  the density accumulation reorder sums).
* A clock budget that runs out stops the loop on the device and reports
  PDEP_ERR_TIMEOUT: nothing waits on anything, so nothing can hang.
* With device buffers chi0_apply only enqueues: the results and the solve
  statistics (iterations, residuals, launches inside graphs) appear once the
  stream is synchronised.
"""
import numpy as np
import pytest

import synthetic

from gpu_common import lib_ready, need_gpu, rel, torch

pytestmark = pytest.mark.gpu


def _pg():
    need_gpu()
    lib_ready()
    import paper_1501_03141_gb300 as pg
    return pg


@pytest.fixture(scope="module")
def tiny():
    return synthetic.make_system("tiny")


def _phi(n, dim, seed=71):
    phi = synthetic.random_vectors(seed, n, dim)
    return phi / np.linalg.norm(phi, axis=1)[:, None]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_chunked_equals_unchunked(tiny, prec):
    pg = _pg()
    p = pg.PDEP_FP64 if prec == "fp64" else pg.PDEP_MIXED
    n = 40
    with pg.Context(tiny, precision=p) as ctx:
        dim = ctx.sizes()["n_pdep_dim"]
        n_r = ctx.sizes()["n_r"]
        phi = _phi(n, dim)
        dn0 = np.empty((n, n_r))
        w0 = ctx.chi0_apply(phi, dn=dn0)
        assert ctx.stats()["chi0_chunks"] == 1
    # 24 MiB of workspace: chi0bar applications of about a dozen perturbations
    with pg.Context(tiny, precision=p, workspace_limit_bytes=24 << 20) as ctx:
        dn1 = np.empty((n, n_r))
        w1 = ctx.chi0_apply(phi, dn=dn1)
        assert ctx.stats()["chi0_chunks"] >= 3
    # chunks change the GEMMs' split-K and hence the rounding: FP64 agrees to
    # rounding, the mixed path to within its FP64 residual bound
    tol = 1e-12 if prec == "fp64" else 1e-8
    assert rel(w1, w0) < tol and rel(dn1, dn0) < tol


def test_chunks_all_written_under_cg_cap(tiny):
    pg = _pg()
    n = 40
    with pg.Context(tiny, cg_max_iter=4) as ctx:
        dim = ctx.sizes()["n_pdep_dim"]
        phi = _phi(n, dim, seed=72)
        w0 = ctx.chi0_apply(phi, allow_unconverged=True)
    with pg.Context(tiny, cg_max_iter=4, workspace_limit_bytes=24 << 20) as ctx:
        out = np.full((n, dim), np.nan)
        with pytest.raises(pg.PdepError) as e:
            ctx.chi0_apply(phi, out=out)
        assert e.value.status == 5
        assert ctx.stats()["chi0_chunks"] >= 3
        out = np.full((n, dim), np.nan)
        ctx.chi0_apply(phi, out=out, allow_unconverged=True)
    assert np.isfinite(out).all() and np.linalg.norm(out, axis=1).min() > 0.0
    assert rel(out, w0) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_equals_host_loop(tiny, prec):
    pg = _pg()
    p = pg.PDEP_FP64 if prec == "fp64" else pg.PDEP_MIXED
    n = 48
    dim = None
    res = {}
    for use_graph in (0, 1):
        # autotune off: the graph is captured from the first call on
        with pg.Context(tiny, precision=p, use_graph=use_graph, autotune=0) as ctx:
            dim = ctx.sizes()["n_pdep_dim"]
            phi = _phi(n, dim, seed=73)
            w = ctx.chi0_apply(phi)
            st = ctx.stats()
            w2 = ctx.chi0_apply(phi)          # second call replays the cached graph
            st2 = ctx.stats()
            res[use_graph] = (w, w2, st, st2)
    (wa, wa2, sa, _), (wb, wb2, sb, sb2) = res[0], res[1]
    assert sa["graph_launches"] == 0 and sb["graph_launches"] >= 1 and sb2["graph_launches"] >= 1
    # the host loop sizes its launches to the active count, the graph to the
    # batch: split-K choices, and so the rounding, may differ
    assert abs(sa["cg_iterations"] - sb["cg_iterations"]) <= 0.02 * sa["cg_iterations"]
    tol = 1e-12 if prec == "fp64" else 1e-8
    # repeated calls differ only by the order of FP64 atomic additions
    assert rel(wb, wa) < tol and rel(wb2, wb) < 1e-12 and rel(wa2, wa) < 1e-12
    # launches inside graphs are counted from the device's step counts
    assert sb["kernel_launches"] >= sa["kernel_launches"] - 4 * sb["graph_launches"]


def test_clock_budget_reports_timeout(tiny):
    pg = _pg()
    n = 16
    for use_graph in (0, 1):
        with pg.Context(tiny, clock_budget_cycles=200, use_graph=use_graph, autotune=0) as ctx:
            dim = ctx.sizes()["n_pdep_dim"]
            phi = _phi(n, dim, seed=74)
            out = np.full((n, dim), np.nan)
            with pytest.raises(pg.PdepError) as e:
                ctx.chi0_apply(phi, out=out)
            assert e.value.status == 7          # PDEP_ERR_TIMEOUT
            assert np.isfinite(out).all()
            st = ctx.stats()
            # the loop stopped after its first step
            assert st["cg_iterations_max"] <= 2
    # the context stays usable: a budget-free context on the same device converges
    with pg.Context(tiny, autotune=0) as ctx:
        ctx.chi0_apply(phi)


def test_device_buffers_enqueue_only(tiny):
    pg = _pg()
    n = 24
    with pg.Context(tiny, precision=pg.PDEP_MIXED, autotune=0) as ctx:
        dim = ctx.sizes()["n_pdep_dim"]
        n_r = ctx.sizes()["n_r"]
        phi = _phi(n, dim, seed=75)
        ref = ctx.chi0_apply(phi)
        dphi = torch.from_numpy(phi).cuda()
        out = torch.empty_like(dphi)
        dn = torch.empty((n, n_r), dtype=torch.float64, device="cuda")
        ctx.chi0_apply(dphi, out=out, dn=dn, sync=False)   # enqueued only
        st = ctx.stats()                                   # synchronises
        assert st["sternheimer_solves"] == n * tiny.n_occ
        assert st["max_cg_residual"] <= 1e-10 and st["cg_iterations"] > 0
        assert st["graph_launches"] >= 1 and st["kernel_launches"] > 0
        # same kernels as the host-buffer call; FP64 atomics may reorder sums
        assert rel(out.cpu().numpy(), ref) < 1e-9
        # sternheimer_solve with device outputs, iteration counts and residuals
        dv = torch.from_numpy(synthetic.random_grid_potentials(76, 2, tiny.grid,
                                                                tiny.cell).reshape(2, -1)).cuda()
        npw = ctx.sizes()["n_pw"]
        dpsi = torch.empty((2, tiny.n_occ, npw), dtype=torch.float64, device="cuda")
        its = torch.empty(2 * tiny.n_occ, dtype=torch.int32, device="cuda")
        res = torch.empty(2 * tiny.n_occ, dtype=torch.float64, device="cuda")
        ctx.sternheimer_solve(dv, dpsi=dpsi, iters=its, resid=res, sync=False)
        torch.cuda.synchronize()
        assert res.max().item() <= 1e-10 and its.min().item() > 0
        h_dpsi, h_its, h_res = ctx.sternheimer_solve(dv.cpu().numpy())
        assert rel(dpsi.cpu().numpy(), h_dpsi) < 1e-9
        assert np.abs(its.cpu().numpy() - h_its).max() <= 1


def test_double_float_refinement_matches_fp64_refinement(tiny):
    """The mixed path's refinement transforms in double-float arithmetic
    (every round: df_refine 1; the first round, FP32 after it: df_refine 2,
    the default) give the same solutions and density responses as FP64
    refinement transforms: each drives the FP64 residual below 1e-10, so they
    agree to within that bound."""
    pg = _pg()
    n = 32
    out = {}
    for df_refine in (0, 1, 2):
        with pg.Context(tiny, precision=pg.PDEP_MIXED, df_refine=df_refine) as ctx:
            dim = ctx.sizes()["n_pdep_dim"]
            phi = _phi(n, dim, seed=77)
            w = ctx.chi0_apply(phi)
            st = ctx.stats()
            assert st["max_cg_residual"] <= 1e-10
            dv = synthetic.random_grid_potentials(78, 2, tiny.grid, tiny.cell).reshape(2, -1)
            dpsi, its, res = ctx.sternheimer_solve(dv)
            assert res.max() <= 1e-10
            out[df_refine] = (w, dpsi, st["refine_rounds_max"])
    for mode in (1, 2):
        e = (rel(out[mode][0], out[0][0]), rel(out[mode][1], out[0][1]))
        print(f"df_refine {mode} vs FP64 refinement: chi0bar phi {e[0]:.2e}, dpsi {e[1]:.2e}, "
              f"rounds {out[mode][2]} vs {out[0][2]}")
        assert e[0] < 1e-8 and e[1] < 1e-8
        assert out[mode][2] <= out[0][2] + 1


def test_fused_transform_matches_three_launch_form(tiny):
    """The inner CG with the fused FP32 H x (one launch, column scratch in
    shared memory) reaches the same FP64-refined solutions as the three-launch
    transforms."""
    pg = _pg()
    n = 32
    out = {}
    for fused in (0, 1):
        with pg.Context(tiny, precision=pg.PDEP_MIXED, fused_hpsi=fused) as ctx:
            dim = ctx.sizes()["n_pdep_dim"]
            phi = _phi(n, dim, seed=79)
            out[fused] = ctx.chi0_apply(phi)
            assert ctx.stats()["max_cg_residual"] <= 1e-10
    assert rel(out[1], out[0]) < 1e-8

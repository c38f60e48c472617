"""A fixed set of library calls whose results the bounds-checked build must
reproduce (used by test_gpu_bounds.py; not a test module).

run_calls() goes through whichever libpdep the process loaded: the normal
build, or libpdep_check.so when PDEP_BOUNDS_CHECK=1 is set before the package
is imported.  Run as a script it saves the results to the .npz path given.

Covered: sphere -> grid and H*psi (FP64 and FP32) on every supported grid
shape (24^3 ... 64^3, 64x64x192), a converged mixed-precision PDEP solve and
a FP64 chi0bar application on the 24^3 workload, short Lanczos chains, and a
mixed chi0bar application of one perturbation on the 48^3 workload.  After
the calls that run no Sternheimer solve the device status word is read with
pdep_sync_status.
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

SHAPES = [
    ((24, 24, 24), (10.0, 10.0, 10.0)),
    ((32, 32, 32), (13.3, 13.3, 13.3)),
    ((40, 40, 40), (16.7, 16.7, 16.7)),
    ((48, 48, 48), (20.0, 20.0, 20.0)),
    ((64, 64, 64), (26.7, 26.7, 26.7)),
    ((64, 64, 192), (20.0, 20.0, 60.0)),
]


def _wells_system(grid, cell, seed=1):
    import synthetic
    rng = np.random.default_rng(seed)
    c, d, w = synthetic.gaussian_wells(rng, 4, cell, (1.0, 3.0), (0.8, 1.5))
    v = synthetic.periodic_gaussian_sum(grid, cell, c, d, w)
    return synthetic.System(name="t", grid=grid, cell=cell, v_r=v, n_occ=2, n_pdep=2, seed=seed)


def run_calls() -> dict:
    import paper_1501_03141_gb300 as pg
    import synthetic
    from paper_1501_03141_gb300 import _abi

    out = {"bounds_checked": np.array(_abi.load().pdep_bounds_checked())}
    for grid, cell in SHAPES:
        tag = "x".join(map(str, grid))
        with pg.Context(_wells_system(grid, cell)) as ctx:
            x = np.random.default_rng(2).standard_normal((3, ctx.sizes()["n_pw"]))
            out[f"grid_{tag}"] = ctx.to_grid(x)
            out[f"h64_{tag}"] = ctx.apply_hamiltonian(x)
            out[f"h32_{tag}"] = ctx.apply_hamiltonian(x, precision=pg.PDEP_MIXED)
            ctx.sync_status()

    tiny = synthetic.make_system("tiny")
    with pg.Context(tiny, precision=pg.PDEP_MIXED) as ctx:
        out["tiny_eig"], _, _ = ctx.pdep_solve()
    with pg.Context(tiny) as ctx:
        dim = ctx.sizes()["n_pdep_dim"]
        n_pw = ctx.sizes()["n_pw"]
        out["tiny_chi0"] = ctx.chi0_apply(synthetic.random_vectors(81, 2, dim))
        rng = np.random.default_rng(82)
        R = rng.standard_normal((3, n_pw))
        L = rng.standard_normal((2, n_pw))
        poles, weights, _, _ = ctx.lanczos(R, 8, L)
        out["tiny_poles"], out["tiny_weights"] = poles, weights
        ctx.sync_status()

    with pg.Context(synthetic.make_system("cube48"), precision=pg.PDEP_MIXED) as ctx:
        phi = synthetic.random_vectors(83, 1, ctx.sizes()["n_pdep_dim"])
        out["cube48_chi0"] = ctx.chi0_apply(phi)
        ctx.sync_status()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_calls())

"""pdep_apply_hamiltonian_noalloc: H*x for callers that cannot allocate.

Callers issuing work during CUDA-graph capture, from host callbacks or under
a pool that owns all device memory cannot call cudaMalloc; this entry point
uses a fixed 16 MiB scratch array instead.  Two calls in a row through the C
ABI must reproduce pdep_apply_hamiltonian (the allocating entry point) to the
tolerance of the H*psi tests.  Named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synthetic

from gpu_common import lib_ready, need_gpu, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n", [("tiny", 5), ("cube48", 103)])
def test_noalloc_matches_allocating_entry_point(name, n):
    need_gpu()
    lib_ready()
    import torch
    import paper_1501_03141_gb300 as pg
    from paper_1501_03141_gb300 import _abi
    s = synthetic.make_system(name)
    s.n_occ = min(s.n_occ, 4)
    with pg.Context(s, gap_min=1e-9) as ctx:
        n_pw = ctx.sizes()["n_pw"]
        x = torch.tensor(np.random.default_rng(7).standard_normal((n, n_pw)), device="cuda")
        ref = ctx.apply_hamiltonian(x.cpu().numpy())
        lib = _abi.load()
        stream = torch.cuda.current_stream().cuda_stream
        outs = []
        for _ in range(2):
            y = torch.full((n, n_pw), np.nan, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            st = lib.pdep_apply_hamiltonian_noalloc(ctx._h, 0, ctypes.c_void_p(x.data_ptr()), n,
                                                    ctypes.c_void_p(y.data_ptr()), stream)
            assert st == _abi.PDEP_OK, lib.pdep_last_error().decode()
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        for y in outs:
            assert rel(y, ref) < 1e-14
        # host buffers are refused (the entry point never stages)
        xh = np.zeros((1, n_pw))
        yh = np.zeros((1, n_pw))
        st = lib.pdep_apply_hamiltonian_noalloc(ctx._h, 0, ctypes.c_void_p(xh.ctypes.data), 1,
                                                ctypes.c_void_p(yh.ctypes.data), stream)
        assert st == _abi.PDEP_ERR_INVALID_ARG

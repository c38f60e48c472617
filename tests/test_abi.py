"""The C-ABI library builds, loads and exports every symbol of include/pdep.h.

No compute call is made: this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pdep.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_03141_gb300 import _abi, build
    build.build(bounds_check=_abi.BOUNDS_CHECK)
    return _abi.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pdep_setup", "chi0_apply", "sternheimer_solve", "pdep_solve",
                     "pdep_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1501_03141_gb300 import _abi
    declared = _declared()
    assert sorted(_abi.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    from paper_1501_03141_gb300 import _abi
    o = _abi.pdep_options()
    lib.pdep_default_options(ctypes.byref(o))
    assert o.precision == _abi.PDEP_FP64 and o.cg_tol == 1e-10
    assert lib.pdep_status_string(_abi.PDEP_ERR_NO_GAP).decode() == "no gap at the Fermi level"
    h = ctypes.c_void_p()
    # a null descriptor is rejected before any device work
    assert lib.pdep_setup(None, 0, None, None, ctypes.byref(h)) == _abi.PDEP_ERR_INVALID_ARG
    assert not h.value


def test_null_context_and_bounds_flag(lib):
    from paper_1501_03141_gb300 import _abi
    assert lib.pdep_sync_status(None, None) == _abi.PDEP_ERR_INVALID_ARG
    assert lib.pdep_bounds_checked() == (1 if _abi.BOUNDS_CHECK else 0)
    assert "bounds" in lib.pdep_status_string(_abi.PDEP_ERR_BOUNDS).decode()


def test_bounds_checked_variant_builds_and_exports():
    """build(bounds_check=True) makes libpdep_check.so, compiled with the index
    tests, exporting the same symbols (loaded side by side, host calls only)."""
    from paper_1501_03141_gb300 import build
    path = build.build(bounds_check=True)
    assert os.path.basename(path) == "libpdep_check.so"
    chk = ctypes.CDLL(path)
    assert chk.pdep_bounds_checked() == 1
    for name in _declared():
        assert hasattr(chk, name), name


def test_python_options_by_name(lib):
    import paper_1501_03141_gb300 as pg
    o = pg.default_options(cg_tol=1e-9, dav_max_iter=7, precision=pg.PDEP_MIXED)
    assert o.cg_tol == 1e-9 and o.dav_max_iter == 7 and o.precision == pg.PDEP_MIXED
    assert o.n_deflate == 16 and o.proj_variant == -1 and o.inner_tol == 1e-5
    # refinement products: double-float in the first round, FP32 after it
    assert o.df_refine == 2
    assert pg.PDEP_MIXED == pg.PDEP_MIXED_TF32 == 1 and pg.PDEP_MIXED_BF16 == 2
    with pytest.raises(KeyError):
        pg.default_options(cg_toll=1e-9)

"""ctypes binding of include/pdep.h (argument marshalling only).

Every function keeps its C name.  Array arguments are numpy arrays (host) or
torch tensors (host or CUDA); the library itself decides how to move them.
Loading fails loudly when libpdep.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
#: PDEP_BOUNDS_CHECK=1 in the environment selects the bounds-checked build
BOUNDS_CHECK = os.environ.get("PDEP_BOUNDS_CHECK", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libpdep_check.so" if BOUNDS_CHECK else "libpdep.so")

PDEP_OK = 0
PDEP_ERR_INVALID_ARG = 1
PDEP_ERR_CUDA = 2
PDEP_ERR_OOM = 3
PDEP_ERR_NO_GAP = 4
PDEP_ERR_NOT_CONVERGED = 5
PDEP_ERR_NONFINITE = 6
PDEP_ERR_TIMEOUT = 7
PDEP_ERR_UNSUPPORTED = 8
PDEP_ERR_BOUNDS = 9

PDEP_FP64 = 0
PDEP_MIXED_TF32 = 1
PDEP_MIXED_BF16 = 2
PDEP_MIXED = PDEP_MIXED_TF32
PDEP_APPLY_DF64 = 3   # pdep_apply_hamiltonian: double-float transforms

PDEP_SCREEN_CHIBAR = 0
PDEP_SCREEN_EPSINV = 1
PDEP_SCREEN_WP = 2

#: every symbol declared in include/pdep.h
EXPORTS = (
    "pdep_default_options", "pdep_setup", "pdep_get_sizes", "pdep_get_occupied",
    "chi0_apply", "sternheimer_solve", "pdep_solve", "pdep_apply_hamiltonian", "pdep_to_grid",
    "pdep_profile", "pdep_destroy", "pdep_status_string", "pdep_last_error",
    "pdep_apply_hamiltonian_noalloc", "pdep_screening_apply", "pdep_lanczos", "pdep_chi0_imag",
    "pdep_chibar_apply", "pdep_sync_status", "pdep_bounds_checked", "pdep_get_stats",
)

PDEP_PROFILE_CLASSES = 17


class pdep_system_desc(ctypes.Structure):
    _fields_ = [
        ("grid", ctypes.c_int * 3),
        ("cell", ctypes.c_double * 3),
        ("ecut", ctypes.c_double),
        ("v_r", ctypes.c_void_p),
        ("n_occ", ctypes.c_int),
        ("n_pdep", ctypes.c_int),
    ]


class pdep_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("cg_tol", ctypes.c_double),
        ("cg_max_iter", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("inner_max_iter", ctypes.c_int),
        ("max_refine", ctypes.c_int),
        ("dav_tol", ctypes.c_double),
        ("dav_max_iter", ctypes.c_int),
        ("dav_subspace_factor", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("gap_min", ctypes.c_double),
        ("setup_tol", ctypes.c_double),
        ("setup_max_iter", ctypes.c_int),
        ("workspace_limit_bytes", ctypes.c_size_t),
        ("n_deflate", ctypes.c_int),
        ("proj_variant", ctypes.c_int),
        ("clock_budget_cycles", ctypes.c_longlong),
        ("autotune", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("df_refine", ctypes.c_int),
        ("fused_hpsi", ctypes.c_int),
    ]


class pdep_stats(ctypes.Structure):
    _fields_ = [
        ("dav_iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("sternheimer_solves", ctypes.c_longlong),
        ("cg_iterations", ctypes.c_longlong),
        ("cg_iterations_max", ctypes.c_int),
        ("refine_rounds_max", ctypes.c_int),
        ("max_cg_residual", ctypes.c_double),
        ("max_dav_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("cg_variant", ctypes.c_int),
        ("proj_variant", ctypes.c_int),
        ("chi0_chunks", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong),
        ("graph_launches", ctypes.c_longlong),
        ("fused_planes", ctypes.c_int),
        ("gemm_shape", ctypes.c_int),
    ]


class pdep_kernel_class(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 24),
        ("launches", ctypes.c_longlong),
        ("ms", ctypes.c_double),
        ("flops", ctypes.c_double),
        ("bytes", ctypes.c_double),
    ]


class pdep_profile_t(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_longlong),
        ("cls", pdep_kernel_class * PDEP_PROFILE_CLASSES),
    ]


_lib = None


def load(path: str = LIB_PATH):
    """Load libpdep.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with paper_1501_03141_gb300.build.build("
            f"bounds_check={BOUNDS_CHECK}) "
            "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.pdep_default_options.argtypes = [ctypes.POINTER(pdep_options)]
    lib.pdep_default_options.restype = None
    lib.pdep_setup.argtypes = [ctypes.POINTER(pdep_system_desc), ip, ctypes.POINTER(pdep_options),
                               vp, ctypes.POINTER(vp)]
    lib.pdep_get_sizes.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip)]
    lib.pdep_get_occupied.argtypes = [vp, ip, vp, vp, vp]
    lib.chi0_apply.argtypes = [vp, ip, vp, ip, vp, vp, vp]
    lib.sternheimer_solve.argtypes = [vp, ip, vp, ip, vp, vp, vp, vp]
    lib.pdep_solve.argtypes = [vp, ip, vp, vp, vp, ctypes.POINTER(pdep_stats), vp]
    lib.pdep_apply_hamiltonian.argtypes = [vp, ip, vp, ip, vp, ip, vp]
    lib.pdep_to_grid.argtypes = [vp, ip, vp, ip, vp, vp]
    lib.pdep_screening_apply.argtypes = [vp, ip, ip, vp, vp, ip, vp, ip, vp, vp]
    lib.pdep_lanczos.argtypes = [vp, ip, vp, ip, ip, vp, ip, vp, vp, vp, vp, vp]
    lib.pdep_chi0_imag.argtypes = [vp, ip, vp, ip, vp, ip, ip, vp, vp, vp]
    lib.pdep_chibar_apply.argtypes = [vp, ip, vp, ip, vp, dp, ip, ctypes.POINTER(ip), vp]
    lib.pdep_apply_hamiltonian_noalloc.argtypes = [vp, ip, vp, ip, vp, vp]
    lib.pdep_apply_hamiltonian_noalloc.restype = ip
    lib.pdep_profile.argtypes = [ip, ctypes.POINTER(pdep_profile_t)]
    lib.pdep_profile.restype = ip
    lib.pdep_destroy.argtypes = [vp]
    lib.pdep_destroy.restype = None
    lib.pdep_status_string.argtypes = [ip]
    lib.pdep_status_string.restype = ctypes.c_char_p
    lib.pdep_last_error.argtypes = []
    lib.pdep_last_error.restype = ctypes.c_char_p
    lib.pdep_sync_status.argtypes = [vp, vp]
    lib.pdep_get_stats.argtypes = [vp, ctypes.POINTER(pdep_stats), vp]
    lib.pdep_bounds_checked.argtypes = []
    for name in ("pdep_setup", "pdep_get_sizes", "pdep_get_occupied", "chi0_apply",
                 "sternheimer_solve", "pdep_solve", "pdep_apply_hamiltonian", "pdep_to_grid",
                 "pdep_screening_apply", "pdep_lanczos", "pdep_chi0_imag",
                 "pdep_chibar_apply", "pdep_sync_status", "pdep_bounds_checked", "pdep_get_stats"):
        getattr(lib, name).restype = ip
    del dp
    _lib = lib
    return lib


class PdepError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.pdep_status_string(status).decode()
        detail = lib.pdep_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")
        self.status = status


def ptr(a) -> int | None:
    """Raw address of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def check(status: int, where: str, allow=(PDEP_OK,)):
    if status not in allow:
        raise PdepError(status, where)
    return status

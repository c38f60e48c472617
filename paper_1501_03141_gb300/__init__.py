"""GB300 PDEP library: Python front end of libpdep.so.

The hot path (Sec. II C of Govoni & Galli, "Large scale GW calculations"):
Davidson diagonalisation of chi0bar = v^{1/2} chi0 v^{1/2} at omega = 0,
where every chi0bar application is a batch of Sternheimer solves.  All the
arithmetic runs in the CUDA kernels of csrc/; this module only marshals
arguments through the C ABI of include/pdep.h.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import PDEP_FP64, PDEP_MIXED, PDEP_MIXED_BF16, PDEP_MIXED_TF32, PdepError  # noqa: F401
from ._abi import PDEP_APPLY_DF64  # noqa: F401
from ._abi import PDEP_SCREEN_CHIBAR, PDEP_SCREEN_EPSINV, PDEP_SCREEN_WP  # noqa: F401

SCREEN_KINDS = {"chibar": PDEP_SCREEN_CHIBAR, "epsinv": PDEP_SCREEN_EPSINV, "wp": PDEP_SCREEN_WP}


def default_options(**kw) -> _abi.pdep_options:
    """pdep_options with the library defaults, overridden by keyword."""
    lib = _abi.load()
    o = _abi.pdep_options()
    lib.pdep_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for the binding
        pass
    return None


def profile_start():
    """Start recording per-kernel-class CUDA-event times (pdep_profile(1))."""
    _abi.check(_abi.load().pdep_profile(1, None), "pdep_profile")


def profile_stop():
    """Stop recording; returns {'launches': n, 'classes': {name: {...}}}."""
    out = _abi.pdep_profile_t()
    _abi.check(_abi.load().pdep_profile(0, ctypes.byref(out)), "pdep_profile")
    classes = {}
    for c in out.cls:
        classes[c.name.decode()] = {"launches": c.launches, "ms": c.ms, "flops": c.flops,
                                    "bytes": c.bytes}
    return {"launches": out.launches, "classes": classes}


class Context:
    """One pdep_ctx holding one or more systems (pdep_setup ... pdep_destroy).

    systems: objects with .grid, .cell, .v_r (float64 array), .n_occ, .n_pdep
    (e.g. synthetic.System).  ecut = 0 selects the alias-free grid rule.
    """

    def __init__(self, systems, options=None, stream=None, ecut=0.0, **opt_kw):
        if not isinstance(systems, (list, tuple)):
            systems = [systems]
        lib = _abi.load()
        self._lib = lib
        self.options = options if options is not None else default_options(**opt_kw)
        n = len(systems)
        desc = (_abi.pdep_system_desc * n)()
        self._keep = []
        for i, s in enumerate(systems):
            v = np.ascontiguousarray(np.asarray(s.v_r, dtype=np.float64))
            self._keep.append(v)
            desc[i].grid[:] = [int(x) for x in s.grid]
            desc[i].cell[:] = [float(x) for x in s.cell]
            desc[i].ecut = float(ecut)
            desc[i].v_r = v.ctypes.data
            desc[i].n_occ = int(s.n_occ)
            desc[i].n_pdep = int(s.n_pdep)
        self.stream = stream
        h = ctypes.c_void_p()
        _abi.check(lib.pdep_setup(desc, n, ctypes.byref(self.options), _stream(stream),
                                  ctypes.byref(h)), "pdep_setup")
        self._h = h
        self.systems = list(systems)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pdep_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- queries -------------------------------------------------------------
    def sizes(self, sys: int = 0):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _abi.check(self._lib.pdep_get_sizes(self._h, sys, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)), "pdep_get_sizes")
        return {"n_pw": a.value, "n_r": b.value, "n_pdep_dim": c.value}

    def occupied(self, sys: int = 0):
        """(psi [n_occ, n_pw], eps [n_occ + 1]) as numpy arrays."""
        sz = self.sizes(sys)
        s = self.systems[sys]
        psi = np.empty((s.n_occ, sz["n_pw"]))
        eps = np.empty(s.n_occ + 1)
        _abi.check(self._lib.pdep_get_occupied(self._h, sys, _abi.ptr(psi), _abi.ptr(eps),
                                               _stream(self.stream)), "pdep_get_occupied")
        return psi, eps

    def sync_status(self):
        """Wait for the context's stream; raise PdepError if a kernel flagged a
        condition (non-finite value, index out of range in a bounds-checked
        build) since the last check, and clear the device status word."""
        _abi.check(self._lib.pdep_sync_status(self._h, _stream(self.stream)), "pdep_sync_status")

    def apply_hamiltonian(self, x, sys: int = 0, precision: int = PDEP_FP64, out=None):
        """H x for sphere vectors x [n, n_pw]."""
        if out is None:
            out = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        _abi.check(self._lib.pdep_apply_hamiltonian(self._h, sys, _abi.ptr(x), int(x.shape[0]),
                                                    _abi.ptr(out), precision,
                                                    _stream(self.stream)), "pdep_apply_hamiltonian")
        return out

    def to_grid(self, x, sys: int = 0, out=None):
        """u(r) = sum_G c(G) e^{iG.r} for sphere vectors x [n, n_pw]; shape [n, n_r]."""
        n_r = self.sizes(sys)["n_r"]
        if out is None:
            out = np.empty((x.shape[0], n_r))
        _abi.check(self._lib.pdep_to_grid(self._h, sys, _abi.ptr(x), int(x.shape[0]), _abi.ptr(out),
                                          _stream(self.stream)), "pdep_to_grid")
        return out

    def stats(self):
        """Statistics of the last hot-path call (pdep_get_stats; synchronises the
        stream and raises PdepError on a pending device condition other than
        'not converged')."""
        st = _abi.pdep_stats()
        r = self._lib.pdep_get_stats(self._h, ctypes.byref(st), _stream(self.stream))
        _abi.check(r, "pdep_get_stats", (_abi.PDEP_OK, _abi.PDEP_ERR_NOT_CONVERGED))
        return {k: getattr(st, k) for k, _ in _abi.pdep_stats._fields_}

    def _finish(self, status, where, allow, bufs, sync):
        """With device buffers only the library call just enqueued the work:
        unless sync is False, wait and read the device status word here."""
        _abi.check(status, where, allow)
        if sync and all(b is None or not isinstance(b, np.ndarray) and b.is_cuda for b in bufs):
            _abi.check(self._lib.pdep_sync_status(self._h, _stream(self.stream)), where, allow)

    # -- hot path ------------------------------------------------------------
    def chi0_apply(self, phi, sys: int = 0, out=None, dn=None, allow_unconverged=False, sync=True):
        """chi0bar phi for phi [n_pert, n_pdep_dim]; returns out (and dn if given).
        With CUDA tensors and sync=False the call only enqueues on the stream."""
        n_pert = int(phi.shape[0])
        if out is None:
            out = np.empty_like(phi) if isinstance(phi, np.ndarray) else phi.new_empty(phi.shape)
        allow = (_abi.PDEP_OK, _abi.PDEP_ERR_NOT_CONVERGED) if allow_unconverged else (_abi.PDEP_OK,)
        r = self._lib.chi0_apply(self._h, sys, _abi.ptr(phi), n_pert, _abi.ptr(out), _abi.ptr(dn),
                                 _stream(self.stream))
        self._finish(r, "chi0_apply", allow, (phi, out, dn), sync)
        return out

    def sternheimer_solve(self, dv, sys: int = 0, dpsi=None, iters=None, resid=None,
                          allow_unconverged=False, sync=True):
        """P_c dpsi for dv [n_pert, n_r]; returns (dpsi [n_pert, n_occ, n_pw], iters, resid)."""
        n_pert = int(dv.shape[0])
        sz = self.sizes(sys)
        s = self.systems[sys]
        if dpsi is None:
            dpsi = np.empty((n_pert, s.n_occ, sz["n_pw"]))
        if iters is None:
            iters = np.empty(n_pert * s.n_occ, dtype=np.int32)
        if resid is None:
            resid = np.empty(n_pert * s.n_occ)
        allow = (_abi.PDEP_OK, _abi.PDEP_ERR_NOT_CONVERGED) if allow_unconverged else (_abi.PDEP_OK,)
        r = self._lib.sternheimer_solve(self._h, sys, _abi.ptr(dv), n_pert, _abi.ptr(dpsi),
                                        _abi.ptr(iters), _abi.ptr(resid), _stream(self.stream))
        self._finish(r, "sternheimer_solve", allow, (dv, dpsi, iters, resid), sync)
        return dpsi, iters, resid

    def pdep_solve(self, sys: int = 0, phi0=None, eigvals=None, eigvecs=None,
                   allow_unconverged=False):
        """Davidson PDEP solve; returns (eigvals, eigvecs, stats dict)."""
        systems = self.systems if sys == -1 else [self.systems[sys]]
        idx = range(len(self.systems)) if sys == -1 else [sys]
        nval = sum(s.n_pdep for s in systems)
        nvec = sum(s.n_pdep * self.sizes(i)["n_pdep_dim"] for s, i in zip(systems, idx))
        if eigvals is None:
            eigvals = np.empty(nval)
        if eigvecs is None:
            eigvecs = np.empty(nvec)
        st = _abi.pdep_stats()
        allow = (_abi.PDEP_OK, _abi.PDEP_ERR_NOT_CONVERGED) if allow_unconverged else (_abi.PDEP_OK,)
        _abi.check(self._lib.pdep_solve(self._h, sys, _abi.ptr(phi0), _abi.ptr(eigvals),
                                        _abi.ptr(eigvecs), ctypes.byref(st),
                                        _stream(self.stream)), "pdep_solve", allow)
        stats = {k: getattr(st, k) for k, _ in _abi.pdep_stats._fields_}
        return eigvals, eigvecs, stats

    def screening_apply(self, kind, eigvals, eigvecs, f, sys: int = 0, out=None):
        """chibar, epsbar^{-1} or W^p at omega = 0 in the PDEP basis applied to f
        [n, n_pdep_dim]; kind is "chibar", "epsinv" or "wp" (or its integer code)."""
        k = SCREEN_KINDS[kind] if isinstance(kind, str) else int(kind)
        n_pdep = int(eigvals.shape[0])
        if out is None:
            out = np.empty_like(f) if isinstance(f, np.ndarray) else f.new_empty(f.shape)
        _abi.check(self._lib.pdep_screening_apply(self._h, sys, k, _abi.ptr(eigvals),
                                                  _abi.ptr(eigvecs), n_pdep, _abi.ptr(f),
                                                  int(f.shape[0]), _abi.ptr(out),
                                                  _stream(self.stream)), "pdep_screening_apply")
        return out

    def lanczos(self, R, n_steps, L=None, sys: int = 0):
        """Lanczos chains of P_c H P_c started on the rows of R [n, n_pw]
        (Sec. II D).  Returns (poles [n, K], weights [n, n_L, K], alpha, beta);
        M_c,LR(omega) ~ sum_k weights[., l, k] / (omega - poles[., k])."""
        n = int(R.shape[0])
        n_L = 0 if L is None else int(L.shape[0])
        poles = np.empty((n, n_steps))
        weights = np.empty((n, n_L, n_steps)) if n_L else None
        alpha = np.empty((n, n_steps))
        beta = np.empty((n, n_steps))
        _abi.check(self._lib.pdep_lanczos(self._h, sys, _abi.ptr(R), n, int(n_steps), _abi.ptr(L),
                                          n_L, _abi.ptr(poles), _abi.ptr(weights), _abi.ptr(alpha),
                                          _abi.ptr(beta), _stream(self.stream)), "pdep_lanczos")
        return poles, weights, alpha, beta

    def chi0_imag(self, phi, nu, n_steps=40, sys: int = 0, with_lambda=True):
        """B(i nu) = phi^T chi0bar(i nu) phi from Lanczos chains and Lambda =
        (1 - B)^{-1} B for phi [n_pdep, n_pdep_dim] and frequencies nu [n_freq]
        (Sec. II B); returns (B, Lambda) of shape [n_freq, n_pdep, n_pdep]."""
        nu = np.ascontiguousarray(np.atleast_1d(np.asarray(nu, dtype=np.float64)))
        n_pdep = int(phi.shape[0])
        B = np.empty((nu.shape[0], n_pdep, n_pdep))
        L = np.empty_like(B) if with_lambda else None
        _abi.check(self._lib.pdep_chi0_imag(self._h, sys, _abi.ptr(phi), n_pdep, _abi.ptr(nu),
                                            int(nu.shape[0]), int(n_steps), _abi.ptr(B),
                                            _abi.ptr(L), _stream(self.stream)), "pdep_chi0_imag")
        return B, L

    def chibar_apply(self, phi, tol=1e-9, max_iter=200, sys: int = 0, out=None):
        """chibar phi with the Hartree-only self-consistent response, by CG on
        (1 - chi0bar) y = phi (Sec. II C); returns (chibar phi, CG iterations)."""
        if out is None:
            out = np.empty_like(phi) if isinstance(phi, np.ndarray) else phi.new_empty(phi.shape)
        it = ctypes.c_int(0)
        _abi.check(self._lib.pdep_chibar_apply(self._h, sys, _abi.ptr(phi), int(phi.shape[0]),
                                               _abi.ptr(out), float(tol), int(max_iter),
                                               ctypes.byref(it), _stream(self.stream)),
                   "pdep_chibar_apply")
        return out, it.value

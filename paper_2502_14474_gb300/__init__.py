"""GB300 (sm_103a) inexact policy iteration for large sparse discounted MDPs.

The compute path is the CUDA library ``libmdp_gb300.so`` behind the C ABI of
``include/mdp.h``; ``capi`` binds it with the same function names.  ``MDP`` is
a small convenience wrapper that keeps the handle and allocates the output
tensors with PyTorch (device memory and streams only).

Problem and method (madupite, "Problem Setting and Solution Methods"):
minimise expected discounted cost on a finite MDP; inexact policy iteration
with GMRES policy evaluation.
"""
from __future__ import annotations

import numpy as np

from . import capi, ingest
from .capi import (MDP_BF16, MDP_F16, MDP_F32, MDP_F64, MDP_FLAG_HOST_INPUT,
                   MDP_FLAG_NO_VALIDATE, MDP_INNER_GMRES, MDP_INNER_RICHARDSON, MDPError,
                   mdp_bellman, mdp_bytes_required, mdp_cancel, mdp_create, mdp_default_opts,
                   mdp_destroy, mdp_info, mdp_last_error, mdp_policy_eval, mdp_profile_enable,
                   mdp_profile_read, mdp_solve, mdp_version)

__all__ = ["MDP", "MDPError", "capi", "ingest", "load", "mdp_create", "mdp_destroy", "mdp_bellman",
           "mdp_policy_eval", "mdp_solve", "mdp_default_opts", "mdp_info", "mdp_bytes_required",
           "mdp_cancel", "mdp_last_error", "mdp_version", "mdp_profile_enable", "mdp_profile_read", "MDP_F32", "MDP_F64", "MDP_BF16",
           "MDP_F16", "MDP_INNER_GMRES", "MDP_INNER_RICHARDSON"]

_STORE = {"f32": MDP_F32, "bf16": MDP_BF16, "f16": MDP_F16}


def load():
    """Load (building if needed) the CUDA library; raises if it is unavailable."""
    return capi.load()


def _torch():
    import torch
    return torch


def _dtype_code(x):
    torch = _torch()
    if isinstance(x, np.ndarray):
        return MDP_F64 if x.dtype == np.float64 else MDP_F32
    if x.dtype == torch.float64:
        return MDP_F64
    if x.dtype == torch.float32:
        return MDP_F32
    raise TypeError(f"unsupported dtype {x.dtype}")


class MDP:
    """A solver handle over a CSR MDP (row r = s*m + a holds P(.|s,a)).

    ``row_ptr`` (int64, n*m+1), ``col`` (int32), ``val`` and ``cost`` (float32
    or float64) are CUDA tensors, or numpy arrays (host input: the library
    copies them in).  ``store`` selects the inner-solve probability precision:
    "f32", "bf16" or "f16" (16-bit copy with per-row renormalisation).
    ``maximize=True`` reads ``cost`` as rewards to maximise; values in and out
    are then in reward terms (see MDP_FLAG_MAXIMIZE in include/mdp.h).
    """

    def __init__(self, n, m, row_ptr, col, val, cost, gamma, store="f32", stream=None,
                 validate=True, device=None, autotune=False, maximize=False):
        torch = _torch()
        self.n, self.m, self.gamma = int(n), int(m), float(gamma)
        host = isinstance(row_ptr, np.ndarray)
        if host:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            val = np.ascontiguousarray(val)
            cost = np.ascontiguousarray(cost)
        else:
            if row_ptr.dtype != torch.int64 or col.dtype != torch.int32:
                raise TypeError("row_ptr must be int64 and col int32")
            for t in (row_ptr, col, val, cost):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("device inputs must be contiguous CUDA tensors")
        self.device = torch.device(device) if device is not None else (
            torch.device("cuda", torch.cuda.current_device()) if host else row_ptr.device)
        flags = (MDP_FLAG_HOST_INPUT if host else 0) | (0 if validate else MDP_FLAG_NO_VALIDATE)
        flags |= capi.MDP_FLAG_AUTOTUNE if autotune else 0
        flags |= capi.MDP_FLAG_MAXIMIZE if maximize else 0
        self.stream = stream
        with torch.cuda.device(self.device):
            self.h = mdp_create(n, m, row_ptr, col, val, _dtype_code(val), cost, _dtype_code(cost),
                                gamma, _STORE[store], stream=self._s(), flags=flags)
        self.store = store
        self.maximize = bool(maximize)

    @classmethod
    def from_csr(cls, mdp, store="f32", device="cuda", host_input=False, validate=True,
                 autotune=False, stream=None, maximize=None):
        """Build from an object with n, m, gamma, row_ptr, col, val, g (numpy);
        ``maximize`` defaults to the object's own ``maximize`` attribute (False
        when it has none)."""
        torch = _torch()
        if maximize is None:
            maximize = bool(getattr(mdp, "maximize", False))
        if host_input:
            return cls(mdp.n, mdp.m, mdp.row_ptr, mdp.col, mdp.val, mdp.g, mdp.gamma, store=store,
                       validate=validate, device=device, autotune=autotune, stream=stream,
                       maximize=maximize)
        dev = torch.device(device)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        return cls(mdp.n, mdp.m, t(mdp.row_ptr), t(mdp.col), t(mdp.val), t(mdp.g), mdp.gamma,
                   store=store, validate=validate, autotune=autotune, stream=stream,
                   maximize=maximize)

    def _s(self):
        torch = _torch()
        return self.stream if self.stream is not None else torch.cuda.current_stream(self.device)

    def close(self):
        if getattr(self, "h", None):
            mdp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        return mdp_info(self.h)

    def profile(self, on=True):
        mdp_profile_enable(self.h, on)

    def profile_read(self) -> dict:
        return mdp_profile_read(self.h)

    def bellman(self, V, want_v=True, want_pi=True, want_r=False):
        """One Bellman backup: returns dict(V=T V, pi, r, res_inf, res_2).

        ``V`` float32 (FP32 path) or float64 (float-float path) CUDA tensor.
        """
        torch = _torch()
        Vo = torch.empty_like(V) if want_v else None
        pi = torch.empty(self.n, dtype=torch.int32, device=V.device) if want_pi else None
        r = torch.empty(self.n, dtype=torch.float32, device=V.device) if want_r else None
        ri, r2 = mdp_bellman(self.h, V, _dtype_code(V), Vo, pi, r, True, stream=self._s())
        return dict(V=Vo, pi=pi, r=r, res_inf=ri, res_2=r2)

    def policy_eval(self, pi, v, tol, restart=30, max_iters=10000, raise_on_not_converged=True):
        """Solve (I - gamma P_pi) v = g_pi in place (v float32/float64 CUDA tensor)."""
        return mdp_policy_eval(self.h, pi, v, _dtype_code(v), tol, restart, max_iters,
                               stream=self._s(), raise_on_not_converged=raise_on_not_converged)

    def solve(self, tol=1e-9, inner_rtol=0.1, restart=30, max_outer=1000, max_inner=10000,
              inner="gmres", cgs2=False, low_precision_inner=None, V_init=None,
              raise_on_not_converged=True, inner_norm="2", s_step=None):
        """Inexact policy iteration; returns (V float64, pi int32, stats dict).
        ``inner``: "gmres" (default), "richardson" (modified policy iteration) or
        "bicgstab".  ``s_step``: GMRES in blocks of s Krylov vectors (0 =
        classical Arnoldi; None = the library default)."""
        torch = _torch()
        o = mdp_default_opts()
        o.tol, o.inner_rtol, o.restart = float(tol), float(inner_rtol), int(restart)
        o.max_outer, o.max_inner = int(max_outer), int(max_inner)
        o.inner = {"gmres": MDP_INNER_GMRES, "richardson": MDP_INNER_RICHARDSON,
                   "bicgstab": capi.MDP_INNER_BICGSTAB}[inner]
        o.cgs2 = 1 if cgs2 else 0
        if low_precision_inner is None:
            low_precision_inner = self.store != "f32"
        o.low_precision_inner = 1 if low_precision_inner else 0
        o.inner_norm = 1 if str(inner_norm) in ("inf", "1") else 0
        if s_step is not None:
            o.s_step = int(s_step)
        if cgs2:
            o.s_step = 0
        V = torch.empty(self.n, dtype=torch.float64, device=self.device)
        pi = torch.empty(self.n, dtype=torch.int32, device=self.device)
        vt = _dtype_code(V_init) if V_init is not None else MDP_F64
        st = mdp_solve(self.h, o, V_init, vt, V, pi, stream=self._s(),
                       raise_on_not_converged=raise_on_not_converged)
        return V, pi, st

"""ctypes binding of the C ABI in include/mdp.h and include/mdp_ingest.h
(argument marshalling only).

Every function below has the name of the C entry point it calls and does no
arithmetic of its own: all work runs in the CUDA library.  Array arguments
are torch tensors (their data pointers are passed) or raw integer addresses.
A non-OK status raises MDPError carrying mdp_last_error().
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MDP_F32, MDP_F64, MDP_BF16, MDP_F16 = 0, 1, 2, 3
MDP_OK = 0
STATUS_NAMES = {0: "MDP_OK", 1: "MDP_ERR_ARG", 2: "MDP_ERR_NOT_STOCHASTIC", 3: "MDP_ERR_OOM",
                4: "MDP_ERR_CUDA", 5: "MDP_ERR_NOT_CONVERGED", 6: "MDP_ERR_TIMEOUT",
                7: "MDP_ERR_CANCELLED", 8: "MDP_ERR_BAD_CSR", 9: "MDP_ERR_NONFINITE"}
MDP_FLAG_HOST_INPUT = 0x1
MDP_FLAG_NO_VALIDATE = 0x2
MDP_FLAG_AUTOTUNE = 0x4
MDP_FLAG_MAXIMIZE = 0x8
MDP_INNER_GMRES, MDP_INNER_RICHARDSON, MDP_INNER_BICGSTAB = 0, 1, 2
MDP_UNSEEN_ERROR, MDP_UNSEEN_SELF_LOOP = 0, 1
MDP_HISTORY = 128

# Every symbol include/*.h declares (checked by the tests).
EXPORTED = sorted(["mdp_create", "mdp_destroy", "mdp_bellman", "mdp_policy_eval",
                   "mdp_default_opts", "mdp_solve", "mdp_info", "mdp_bytes_required", "mdp_cancel",
                   "mdp_last_error", "mdp_version", "mdp_profile_enable", "mdp_profile_read",
                   "mdp_bellman_noalloc", "mdp_batch_solve", "mdp_pool_trim", "mdp_last_cycle",
                   "mdp_batch_solve_fused",
                   "mdp_csr_from_functions", "mdp_csr_from_rows", "mdp_csr_from_samples",
                   "mdp_csr_read_petsc",
                   "mdp_csr_write_petsc", "mdp_csr_free"])

PROF_KINDS = ["bellman_f32", "bellman_ff", "policy_residual", "arnoldi_spmv", "arnoldi_ortho",
              "gmres_update", "richardson", "other", "arnoldi_dots", "bicgstab_spmv", "block_gram",
              "block_update"]


class MDPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        self.status_name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.status_name}: {msg}")


class mdp_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_rtol", ctypes.c_double),
                ("restart", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("max_inner", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("cgs2", ctypes.c_int32), ("low_precision_inner", ctypes.c_int32),
                ("inner_norm", ctypes.c_int32), ("s_step", ctypes.c_int32)]


class mdp_solve_stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("bellman_sweeps", ctypes.c_int32), ("policy_sweeps", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("n_history", ctypes.c_int32),
                ("residual_inf", ctypes.c_double), ("transitions", ctypes.c_double),
                ("residual_history", ctypes.c_double * MDP_HISTORY),
                ("inner_history", ctypes.c_int32 * MDP_HISTORY)]

    def as_dict(self):
        k = self.n_history
        return dict(outer_iters=self.outer_iters, inner_iters=self.inner_iters,
                    bellman_sweeps=self.bellman_sweeps, policy_sweeps=self.policy_sweeps,
                    converged=bool(self.converged), residual_inf=self.residual_inf,
                    transitions=self.transitions,
                    residual_history=list(self.residual_history[:k]),
                    inner_history=list(self.inner_history[:max(0, self.outer_iters)]))


class mdp_eval_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("policy_sweeps", ctypes.c_int32),
                ("residual_2", ctypes.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, cycles=self.cycles, converged=bool(self.converged),
                    policy_sweeps=self.policy_sweeps, residual_2=self.residual_2)


class mdp_info_t(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int64), ("n_rows", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_actions", ctypes.c_int32), ("vec_width", ctypes.c_int32),
                ("uniform_len", ctypes.c_int32), ("idx64", ctypes.c_int32),
                ("band", ctypes.c_int64), ("has_low_precision", ctypes.c_int32),
                ("store_t", ctypes.c_int32), ("device_bytes", ctypes.c_size_t),
                ("gamma", ctypes.c_double), ("maximize", ctypes.c_int32),
                ("window", ctypes.c_int32), ("ff_screen", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


MDP_MAX_RESTART = 64


class mdp_gmres_cycle_t(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("pad", ctypes.c_int32), ("beta", ctypes.c_double),
                ("est", ctypes.c_double),
                ("H", ctypes.c_double * ((MDP_MAX_RESTART + 1) * MDP_MAX_RESTART)),
                ("y", ctypes.c_double * MDP_MAX_RESTART)]

    def as_dict(self):
        import numpy as np
        J = self.J
        H = np.ctypeslib.as_array(self.H).reshape(MDP_MAX_RESTART, MDP_MAX_RESTART + 1).T
        return {"J": J, "beta": self.beta, "est": self.est,
                "H": np.triu(np.array(H[:J + 1, :J]), -1), "y": np.array(self.y[:J])}


class mdp_profile_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 12), ("skipped", ctypes.c_int64 * 12),
                ("ms", ctypes.c_double * 12), ("bytes", ctypes.c_double * 12),
                ("total_launches", ctypes.c_int64), ("p50_ms", ctypes.c_double * 12),
                ("p99_ms", ctypes.c_double * 12)]

    def as_dict(self):
        kinds = {}
        for i, name in enumerate(PROF_KINDS):
            if name.startswith("unused"):
                continue
            kinds[name] = dict(launches=self.launches[i], skipped=self.skipped[i],
                               ms=self.ms[i], bytes=self.bytes[i], p50_ms=self.p50_ms[i],
                               p99_ms=self.p99_ms[i])
        return dict(kinds=kinds, total_launches=self.total_launches)


class mdp_host_csr(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int64), ("n_actions", ctypes.c_int32),
                ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("cost", ctypes.c_void_p), ("owned", ctypes.c_int32)]


MDP_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
MDP_ROW_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                              ctypes.c_void_p)
MDP_COST_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libmdp_gb300.so (building it with nvcc first if it is missing).

    Raises if the library cannot be built or loaded: there is no fallback.
    """
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; build it with "
                               "paper_2502_14474_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P, I32, I64, D, U64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_uint64)
        lib.mdp_create.argtypes = [ctypes.POINTER(P), I64, I32, P, P, P, ctypes.c_int, P,
                                   ctypes.c_int, D, ctypes.c_int, P, U64]
        lib.mdp_create.restype = ctypes.c_int
        lib.mdp_destroy.argtypes = [P]
        lib.mdp_destroy.restype = None
        lib.mdp_bellman.argtypes = [P, P, ctypes.c_int, P, P, P, ctypes.POINTER(D),
                                    ctypes.POINTER(D), P]
        lib.mdp_bellman.restype = ctypes.c_int
        lib.mdp_policy_eval.argtypes = [P, P, P, ctypes.c_int, D, I32, I32,
                                        ctypes.POINTER(mdp_eval_stats), P]
        lib.mdp_policy_eval.restype = ctypes.c_int
        lib.mdp_default_opts.argtypes = [ctypes.POINTER(mdp_solve_opts)]
        lib.mdp_default_opts.restype = None
        lib.mdp_solve.argtypes = [P, ctypes.POINTER(mdp_solve_opts), P, ctypes.c_int, P, P,
                                  ctypes.POINTER(mdp_solve_stats), P]
        lib.mdp_solve.restype = ctypes.c_int
        lib.mdp_info.argtypes = [P, ctypes.POINTER(mdp_info_t)]
        lib.mdp_info.restype = ctypes.c_int
        lib.mdp_last_cycle.argtypes = [P, ctypes.POINTER(mdp_gmres_cycle_t)]
        lib.mdp_last_cycle.restype = ctypes.c_int
        lib.mdp_bytes_required.argtypes = [I64, I32, I64, ctypes.c_int, ctypes.c_int, I32]
        lib.mdp_bytes_required.restype = ctypes.c_size_t
        lib.mdp_cancel.argtypes = [P]
        lib.mdp_cancel.restype = None
        lib.mdp_profile_enable.argtypes = [P, ctypes.c_int]
        lib.mdp_profile_enable.restype = ctypes.c_int
        lib.mdp_profile_read.argtypes = [P, ctypes.POINTER(mdp_profile_t)]
        lib.mdp_profile_read.restype = ctypes.c_int
        lib.mdp_bellman_noalloc.argtypes = [I64, I32, P, P, P, P, D, P, P, P, P,
                                            ctypes.POINTER(D), ctypes.POINTER(D), P]
        lib.mdp_bellman_noalloc.restype = ctypes.c_int
        lib.mdp_batch_solve.argtypes = [P, I32, ctypes.POINTER(mdp_solve_opts), P, P,
                                        ctypes.POINTER(mdp_solve_stats), P, I32]
        lib.mdp_batch_solve.restype = ctypes.c_int
        lib.mdp_batch_solve_fused.argtypes = [P, I32, ctypes.POINTER(mdp_solve_opts), P, P,
                                              ctypes.POINTER(mdp_solve_stats),
                                              ctypes.POINTER(ctypes.c_int), P]
        lib.mdp_batch_solve_fused.restype = ctypes.c_int
        lib.mdp_pool_trim.argtypes = [I32, U64, ctypes.POINTER(U64)]
        lib.mdp_pool_trim.restype = ctypes.c_int
        HP = ctypes.POINTER(mdp_host_csr)
        lib.mdp_csr_from_functions.argtypes = [I64, I32, MDP_ROW_FN, MDP_COST_FN, P, I32,
                                               MDP_ALLOC_FN, P, HP]
        lib.mdp_csr_from_functions.restype = ctypes.c_int
        lib.mdp_csr_from_rows.argtypes = [I64, I32, P, P, P, P, I32, MDP_ALLOC_FN, P, HP]
        lib.mdp_csr_from_rows.restype = ctypes.c_int
        lib.mdp_csr_from_samples.argtypes = [I64, I32, I64, P, P, P, P, I32, D, I32,
                                             MDP_ALLOC_FN, P, HP]
        lib.mdp_csr_from_samples.restype = ctypes.c_int
        lib.mdp_csr_read_petsc.argtypes = [ctypes.c_char_p, ctypes.c_char_p, I32, MDP_ALLOC_FN,
                                           P, HP]
        lib.mdp_csr_read_petsc.restype = ctypes.c_int
        lib.mdp_csr_write_petsc.argtypes = [HP, ctypes.c_char_p, ctypes.c_char_p]
        lib.mdp_csr_write_petsc.restype = ctypes.c_int
        lib.mdp_csr_free.argtypes = [HP]
        lib.mdp_csr_free.restype = None
        lib.mdp_last_error.argtypes = []
        lib.mdp_last_error.restype = ctypes.c_char_p
        lib.mdp_version.argtypes = []
        lib.mdp_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _ptr(x):
    """Data pointer of a tensor / numpy array, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int):
    if rc != MDP_OK:
        msg = load().mdp_last_error().decode(errors="replace")
        raise MDPError(rc, msg)


def mdp_last_error() -> str:
    return load().mdp_last_error().decode(errors="replace")


def mdp_version() -> str:
    return load().mdp_version().decode()


def mdp_create(n_states, n_actions, row_ptr, col, val, val_t, cost, cost_t, gamma, store_t,
               stream=None, flags=0):
    """Returns the handle (an integer address)."""
    h = ctypes.c_void_p()
    rc = load().mdp_create(ctypes.byref(h), int(n_states), int(n_actions), _ptr(row_ptr),
                           _ptr(col), _ptr(val), int(val_t), _ptr(cost), int(cost_t), float(gamma),
                           int(store_t), _stream(stream), int(flags))
    _check(rc)
    return h.value


def mdp_destroy(h):
    if h:
        load().mdp_destroy(h)


def mdp_bellman(h, V_in, v_t, V_out=None, pi_out=None, r_out=None, want_norms=True,
                stream=None):
    """Returns (res_inf, res_2) when want_norms, else None."""
    ri, r2 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().mdp_bellman(h, _ptr(V_in), int(v_t), _ptr(V_out), _ptr(pi_out), _ptr(r_out),
                            ctypes.byref(ri) if want_norms else None,
                            ctypes.byref(r2) if want_norms else None, _stream(stream))
    _check(rc)
    return (ri.value, r2.value) if want_norms else None


def mdp_policy_eval(h, pi, v_inout, v_t, tol, restart=30, max_iters=10000, stream=None,
                    raise_on_not_converged=True):
    st = mdp_eval_stats()
    rc = load().mdp_policy_eval(h, _ptr(pi), _ptr(v_inout), int(v_t), float(tol), int(restart),
                                int(max_iters), ctypes.byref(st), _stream(stream))
    if rc != MDP_OK and not (rc == 5 and not raise_on_not_converged):
        _check(rc)
    d = st.as_dict()
    d["status"] = STATUS_NAMES.get(rc, rc)
    return d


def mdp_default_opts() -> mdp_solve_opts:
    o = mdp_solve_opts()
    load().mdp_default_opts(ctypes.byref(o))
    return o


def mdp_solve(h, opts=None, V_init=None, vinit_t=MDP_F64, V_out=None, pi_out=None, stream=None,
              raise_on_not_converged=True):
    st = mdp_solve_stats()
    rc = load().mdp_solve(h, ctypes.byref(opts) if opts is not None else None, _ptr(V_init),
                          int(vinit_t), _ptr(V_out), _ptr(pi_out), ctypes.byref(st),
                          _stream(stream))
    if rc != MDP_OK and not (rc == 5 and not raise_on_not_converged):
        _check(rc)
    d = st.as_dict()
    d["status"] = STATUS_NAMES.get(rc, rc)
    return d


def mdp_info(h) -> dict:
    info = mdp_info_t()
    _check(load().mdp_info(h, ctypes.byref(info)))
    return info.as_dict()


def mdp_last_cycle(h) -> dict:
    """The last finished GMRES cycle: J, beta, est, H ((J+1) x J, before the Givens
    rotations) and the least-squares solution y."""
    c = mdp_gmres_cycle_t()
    _check(load().mdp_last_cycle(h, ctypes.byref(c)))
    return c.as_dict()


def mdp_bytes_required(n_states, n_actions, nnz, val_t=MDP_F32, store_t=MDP_F32, restart=30):
    return int(load().mdp_bytes_required(int(n_states), int(n_actions), int(nnz), int(val_t),
                                         int(store_t), int(restart)))


def mdp_pool_trim(device: int = 0, keep_bytes: int = 0) -> int:
    """Release device memory cached by the library's pool on `device` down to
    keep_bytes; returns the bytes the pool still reserves."""
    out = ctypes.c_uint64(0)
    _check(load().mdp_pool_trim(int(device), int(keep_bytes), ctypes.byref(out)))
    return int(out.value)


def mdp_cancel(h):
    load().mdp_cancel(h)


def mdp_profile_enable(h, on=True):
    _check(load().mdp_profile_enable(h, 1 if on else 0))


def mdp_profile_read(h) -> dict:
    p = mdp_profile_t()
    _check(load().mdp_profile_read(h, ctypes.byref(p)))
    return p.as_dict()


def mdp_bellman_noalloc(n_states, n_actions, row_ptr, col, val, cost, gamma, V_in, V_out=None,
                        pi_out=None, r_out=None, stream=None):
    """FP32 Bellman backup on a caller's CSR without any allocation; returns
    (res_inf, res_2).  See include/mdp.h for the scratch limit and sharing."""
    ri, r2 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().mdp_bellman_noalloc(int(n_states), int(n_actions), _ptr(row_ptr), _ptr(col),
                                    _ptr(val), _ptr(cost), float(gamma), _ptr(V_in), _ptr(V_out),
                                    _ptr(pi_out), _ptr(r_out), ctypes.byref(ri),
                                    ctypes.byref(r2), _stream(stream))
    _check(rc)
    return ri.value, r2.value


def mdp_batch_solve(handles, V_outs, pi_outs=None, opts=None, n_streams=8,
                    raise_on_error=True):
    """Solve independent MDPs concurrently; returns (per-MDP stats dicts, statuses)."""
    count = len(handles)
    H = (ctypes.c_void_p * max(count, 1))(*handles)
    Vp = (ctypes.c_void_p * max(count, 1))(*[_ptr(v) for v in V_outs])
    Pp = (ctypes.c_void_p * max(count, 1))(*[_ptr(p) for p in pi_outs]) if pi_outs else None
    st = (mdp_solve_stats * max(count, 1))()
    status = (ctypes.c_int * max(count, 1))()
    rc = load().mdp_batch_solve(H, count, ctypes.byref(opts) if opts is not None else None, Vp,
                                Pp, st, status, int(n_streams))
    if rc != MDP_OK and raise_on_error:
        _check(rc)
    return [st[i].as_dict() for i in range(count)], [STATUS_NAMES.get(status[i], status[i])
                                                     for i in range(count)]


def mdp_batch_solve_fused(handles, V_outs, pi_outs=None, opts=None, stream=None,
                          raise_on_error=True):
    """Solve independent MDPs with every solve phase of all of them in one launch;
    returns (per-MDP stats dicts, statuses)."""
    count = len(handles)
    H = (ctypes.c_void_p * max(count, 1))(*handles)
    Vp = (ctypes.c_void_p * max(count, 1))(*[_ptr(v) for v in V_outs])
    Pp = (ctypes.c_void_p * max(count, 1))(*[_ptr(p) for p in pi_outs]) if pi_outs else None
    st = (mdp_solve_stats * max(count, 1))()
    status = (ctypes.c_int * max(count, 1))()
    rc = load().mdp_batch_solve_fused(H, count,
                                      ctypes.byref(opts) if opts is not None else None, Vp, Pp,
                                      st, status, _stream(stream))
    if rc != MDP_OK and raise_on_error:
        _check(rc)
    return [st[i].as_dict() for i in range(count)], [STATUS_NAMES.get(status[i], status[i])
                                                     for i in range(count)]


def _path(p):
    return None if p is None else os.fsencode(p)


def _alloc_fn(alloc):
    return alloc if alloc is not None else MDP_ALLOC_FN()


def mdp_csr_from_functions(n_states, n_actions, row_fn, cost_fn, threads=1, alloc=None):
    """row_fn / cost_fn: MDP_ROW_FN / MDP_COST_FN objects; alloc: an MDP_ALLOC_FN
    or None (malloc; release with mdp_csr_free).  Returns the mdp_host_csr."""
    out = mdp_host_csr()
    _check(load().mdp_csr_from_functions(int(n_states), int(n_actions), row_fn, cost_fn, None,
                                         int(threads), _alloc_fn(alloc), None, ctypes.byref(out)))
    return out


def mdp_csr_from_rows(n_states, n_actions, offsets, col, prob, cost, threads=0, alloc=None):
    """offsets int64[n*m+1], col int32, prob and cost float64 arrays."""
    out = mdp_host_csr()
    _check(load().mdp_csr_from_rows(int(n_states), int(n_actions), _ptr(offsets), _ptr(col),
                                    _ptr(prob), _ptr(cost), int(threads), _alloc_fn(alloc), None,
                                    ctypes.byref(out)))
    return out


def mdp_csr_from_samples(n_states, n_actions, s, a, s_next, c=None, unseen=MDP_UNSEEN_ERROR,
                         unseen_cost=0.0, threads=0, alloc=None):
    """s, s_next int64 and a int32 arrays (c float64 or None) of one length."""
    out = mdp_host_csr()
    _check(load().mdp_csr_from_samples(int(n_states), int(n_actions), len(s), _ptr(s), _ptr(a),
                                       _ptr(s_next), _ptr(c), int(unseen), float(unseen_cost),
                                       int(threads), _alloc_fn(alloc), None, ctypes.byref(out)))
    return out


def mdp_csr_read_petsc(p_path, g_path=None, threads=0, alloc=None):
    out = mdp_host_csr()
    _check(load().mdp_csr_read_petsc(_path(p_path), _path(g_path), int(threads),
                                     _alloc_fn(alloc), None, ctypes.byref(out)))
    return out


def mdp_csr_write_petsc(csr, p_path, g_path=None):
    _check(load().mdp_csr_write_petsc(ctypes.byref(csr), _path(p_path), _path(g_path)))


def mdp_csr_free(csr):
    load().mdp_csr_free(ctypes.byref(csr))

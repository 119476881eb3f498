"""FP64 CPU oracle for the discounted-MDP hot path.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference the GPU
solver is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library (``paper_2502_14474_gb300``) and never imports it.

What it computes (madupite, "Problem Setting and Solution Methods": infinite-
horizon discounted MDPs with finite state and action spaces, minimising the
expected discounted cost; solution by policy iteration and its inexact
variants, Bertsekas 2007):

* ``bellman``            one application of the Bellman operator T with the
                         greedy (lowest-index argmin) policy, the Q values and
                         the Q-gap (C, FP64, ``oracle.c``).
* ``policy_apply``       one application of T_pi (C, FP64).
* ``value_iteration``    V_{k+1} = T V_k from V_0 = 0 until the contraction
                         bound guarantees ||V - V*||_inf <= tol.
* ``policy_evaluate``    V_pi = (I - gamma P_pi)^{-1} g_pi by dense LU with
                         partial pivoting (LAPACK ``gesv`` through numpy).
* ``policy_iteration``   exact policy iteration with dense LU evaluation.
* ``certificate``        ||T V - V||_inf on the given states and the bound
                         ||V - V*||_inf <= ||T V - V||_inf / (1 - gamma).

Every function is pinned by tests against closed forms, brute force over all
deterministic policies on tiny MDPs, and the contraction / monotonicity
invariants of T (``tests/test_oracle.py``).
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, OpenMP over states; the sums stay sequential)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stamp = os.path.join(_OUT_DIR, "HOST_ARCH")
    if not (os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()):
        force = True
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            lib.oracle_bellman.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, f64, vp, vp, vp, vp,
                                           vp]
            lib.oracle_bellman.restype = None
            lib.oracle_policy_apply.argtypes = [i64, i32, vp, vp, vp, vp, vp, vp, f64, vp, vp, vp]
            lib.oracle_policy_apply.restype = None
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _vals(x):
    """(float32 pointer source, float64 pointer source) for a stored array."""
    x = np.ascontiguousarray(x)
    if x.dtype == np.float32:
        return x, None
    return None, np.ascontiguousarray(x, dtype=np.float64)


def _csr(mdp):
    row_ptr = np.ascontiguousarray(mdp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(mdp.col, dtype=np.int32)
    v32, v64 = _vals(mdp.val)
    g32, g64 = _vals(mdp.g)
    return row_ptr, col, v32, v64, g32, g64


def bellman(mdp, V, want_q: bool = False, want_gap: bool = False):
    """T V, the greedy policy, and optionally Q and the Q-gap, on mdp's states.

    ``V`` is the full value vector (length ``mdp.n``).  Returns
    ``(TV, pi)`` or ``(TV, pi, Q, gap)`` with the optional entries None when not
    requested.  Q has shape (n_local, m).
    """
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.shape != (mdp.n,):
        raise ValueError("V must have one entry per state")
    nl = mdp.n_local
    row_ptr, col, v32, v64, g32, g64 = _csr(mdp)
    TV = np.empty(nl, dtype=np.float64)
    pi = np.empty(nl, dtype=np.int32)
    Q = np.empty(nl * mdp.m, dtype=np.float64) if want_q else None
    gap = np.empty(nl, dtype=np.float64) if want_gap else None
    lib.oracle_bellman(nl, mdp.m, _p(row_ptr), _p(col), _p(v32), _p(v64), _p(g32), _p(g64),
                       float(mdp.gamma), _p(V), _p(TV), _p(pi), _p(Q), _p(gap))
    if want_q or want_gap:
        return TV, pi, (Q.reshape(nl, mdp.m) if Q is not None else None), gap
    return TV, pi


def policy_apply(mdp, pi, V):
    """T_pi V on mdp's states: g(s, pi(s)) + gamma * sum_s' P(s'|s, pi(s)) V(s')."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.float64)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    if V.shape != (mdp.n,) or pi.shape != (mdp.n_local,):
        raise ValueError("shape mismatch")
    if pi.size and (pi.min() < 0 or pi.max() >= mdp.m):
        raise ValueError("action out of range")
    row_ptr, col, v32, v64, g32, g64 = _csr(mdp)
    out = np.empty(mdp.n_local, dtype=np.float64)
    lib.oracle_policy_apply(mdp.n_local, mdp.m, _p(row_ptr), _p(col), _p(v32), _p(v64), _p(g32),
                            _p(g64), float(mdp.gamma), _p(pi), _p(V), _p(out))
    return out


def greedy(mdp, V):
    return bellman(mdp, V)[1]


def value_iteration(mdp, tol: float, V0=None, max_iter: int = 10**7):
    """Value iteration V_{k+1} = T V_k (the Bellman fixed-point iteration).

    Stops once ||V_{k+1} - V_k||_inf <= tol (1 - gamma) / gamma, which bounds
    ||V_{k+1} - V*||_inf <= tol by the gamma-contraction of T.  Returns
    (V, pi, iterations, history of ||V_{k+1} - V_k||_inf).
    """
    if mdp.n_local != mdp.n:
        raise ValueError("value iteration needs the whole MDP")
    g = float(mdp.gamma)
    V = np.zeros(mdp.n) if V0 is None else np.array(V0, dtype=np.float64)
    stop = tol * (1.0 - g) / g if g > 0 else 0.0
    hist = []
    for it in range(1, max_iter + 1):
        TV, pi = bellman(mdp, V)
        d = float(np.max(np.abs(TV - V))) if mdp.n else 0.0
        hist.append(d)
        V = TV
        if d <= stop:
            return V, greedy(mdp, V), it, hist
    raise RuntimeError("value iteration did not converge")


def policy_matrix(mdp, pi):
    """Dense P_pi (n x n) and g_pi (n) of a deterministic policy."""
    if mdp.n_local != mdp.n:
        raise ValueError("needs the whole MDP")
    n, m = mdp.n, mdp.m
    pi = np.asarray(pi, dtype=np.int64)
    rows = np.arange(n, dtype=np.int64) * m + pi
    P = np.zeros((n, n), dtype=np.float64)
    for s in range(n):
        b, e = mdp.row_ptr[rows[s]], mdp.row_ptr[rows[s] + 1]
        P[s, mdp.col[b:e]] = mdp.val[b:e].astype(np.float64)
    gp = mdp.g.astype(np.float64)[rows]
    return P, gp


def policy_evaluate(mdp, pi):
    """V_pi solving (I - gamma P_pi) V = g_pi by dense LU with partial pivoting."""
    P, gp = policy_matrix(mdp, pi)
    A = np.eye(mdp.n) - float(mdp.gamma) * P
    return np.linalg.solve(A, gp)


def policy_iteration(mdp, max_iter: int = 1000):
    """Exact policy iteration (Bertsekas 2007) with dense LU evaluation.

    pi_0 = greedy(0) (the lowest-index argmin of g); evaluate V_pi exactly;
    improve greedily, keeping pi(s) whenever its Q is within 1e-14 |Q| of the
    minimum so that rounding cannot make the loop cycle; stop when the policy
    is stable.  The returned policy is the plain lowest-index greedy policy of
    the final V.  Returns (V, pi, iterations, list of V_pi per iteration).
    """
    pi = greedy(mdp, np.zeros(mdp.n))
    history = []
    for it in range(1, max_iter + 1):
        V = policy_evaluate(mdp, pi)
        history.append(V)
        _, new_pi, Q, _ = bellman(mdp, V, want_q=True)
        qmin = Q.min(axis=1)
        keep = Q[np.arange(mdp.n), pi] <= qmin + 1e-14 * np.abs(qmin)
        new_pi = np.where(keep, pi, new_pi).astype(np.int32)
        if np.array_equal(new_pi, pi):
            return V, greedy(mdp, V), it, history
        pi = new_pi
    raise RuntimeError("policy iteration did not converge")


def certificate(mdp, V):
    """Bellman residual of V on mdp's states and the implied error bound.

    Returns dict(res_inf = ||T V - V||_inf over the local states,
    bound = res_inf / (1 - gamma)  (>= ||V - V*||_inf when the states are all
    of them), TV, pi, gap).
    """
    V = np.ascontiguousarray(V, dtype=np.float64)
    TV, pi, _, gap = bellman(mdp, V, want_gap=True)
    loc = V[mdp.s0:mdp.s0 + mdp.n_local]
    res = float(np.max(np.abs(TV - loc))) if mdp.n_local else 0.0
    return dict(res_inf=res, bound=res / (1.0 - float(mdp.gamma)), TV=TV, pi=pi, gap=gap)

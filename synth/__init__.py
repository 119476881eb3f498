"""Seeded synthetic MDP workloads shared by the oracle, the tests and the bench.

This module only draws inputs: the CSR transition matrix ``P`` (``n*m`` rows,
row ``r = s*m + a``, successors ascending) and the stage costs ``g``.  It holds
none of the solver's arithmetic.  The C code in ``synth.c`` is compiled with
gcc on first use (OpenMP over rows; output independent of the thread count).

Workloads (seeded; shapes of the paper's problem class, finite discounted
MDPs with sparse transitions):

* ``random_sparse``  n states, m actions, k successors per row drawn uniformly
  without replacement from all states, Dirichlet(alpha) probabilities,
  g ~ U[0, 1].  Optional per-row successor range [k_min, k_max].
* ``banded``         as above but successors drawn from the clipped window
  [s - band, s + band].
* ``grid_world``     W x H grid, actions N/E/S/W/stay, p_int to the intended
  cell, p_oth to each other stencil cell, reflecting walls, cost 1 except 0 at
  goal cells.
* ``uneven_batch_params``  the per-MDP parameters of a batch of independent
  random MDPs of uneven size.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library (gcc, -O2, OpenMP)."""
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
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, f64, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.synth_philox4x32_10.argtypes = [vp, vp, vp]
            lib.synth_philox4x32_10.restype = None
            lib.synth_random_row_ptr.argtypes = [i64, i64, i32, i32, i32, u64, vp]
            lib.synth_random_row_ptr.restype = i64
            lib.synth_random_fill.argtypes = [i64, i64, i64, i32, i64, f64, u64, vp, vp, vp,
                                              i32, vp, i32]
            lib.synth_random_fill.restype = ctypes.c_int
            lib.synth_grid_goals.argtypes = [i64, i64, i32, u64, vp]
            lib.synth_grid_goals.restype = None
            lib.synth_grid_fill.argtypes = [i64, i64, i64, i64, f64, f64, vp, i32, i32, vp, vp,
                                            vp, i32, vp, i32]
            lib.synth_grid_fill.restype = i64
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


@dataclasses.dataclass
class CSRMDP:
    """Host CSR MDP over the states [s0, s0 + n_local) of an n-state MDP.

    ``row_ptr`` is local (starts at 0) with ``n_local*m + 1`` int64 entries;
    ``col`` holds global state indices (int32); ``val`` and ``g`` are float32
    or float64.
    """

    n: int
    m: int
    gamma: float
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    g: np.ndarray
    s0: int = 0
    name: str = ""

    @property
    def n_local(self) -> int:
        return (len(self.row_ptr) - 1) // self.m

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def rows(self) -> int:
        return len(self.row_ptr) - 1


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (exposed for known-answer tests)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return [int(x) for x in out]


def random_sparse(n: int, m: int, k: int, alpha: float, gamma: float, seed: int, *,
                  band: int = -1, k_max: int | None = None, s0: int = 0, s1: int | None = None,
                  dtype=np.float64, name: str = "") -> CSRMDP:
    """Random (band < 0) or banded MDP; states [s0, s1) of the n-state instance."""
    lib = _load()
    s1 = n if s1 is None else s1
    k_min = k
    k_max = k if k_max is None else k_max
    if not (0 <= s0 <= s1 <= n) or m < 1 or k_min < 1 or k_max < k_min:
        raise ValueError("bad generator arguments")
    rows = (s1 - s0) * m
    row_ptr = np.empty(rows + 1, dtype=np.int64)
    nnz = lib.synth_random_row_ptr(s0, s1, m, k_min, k_max, seed, _ptr(row_ptr))
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=dtype)
    g = np.empty(rows, dtype=dtype)
    is64 = 1 if np.dtype(dtype) == np.float64 else 0
    rc = lib.synth_random_fill(n, s0, s1, m, band, alpha, seed, _ptr(row_ptr), _ptr(col),
                               _ptr(val), is64, _ptr(g), is64)
    if rc != 0:
        raise ValueError("more successors requested than the window holds")
    return CSRMDP(n=n, m=m, gamma=gamma, row_ptr=row_ptr, col=col, val=val, g=g, s0=s0,
                  name=name)


def banded(n: int, m: int, k: int, band: int, alpha: float, gamma: float, seed: int,
           **kw) -> CSRMDP:
    return random_sparse(n, m, k, alpha, gamma, seed, band=band, **kw)


def grid_goals(W: int, H: int, n_goals: int, seed: int) -> np.ndarray:
    lib = _load()
    goals = np.empty(n_goals, dtype=np.int64)
    lib.synth_grid_goals(W, H, n_goals, seed, _ptr(goals))
    return goals


def grid_world(W: int, H: int, gamma: float, seed: int, *, p_int: float = 0.8,
               p_oth: float = 0.05, n_goals: int = 16, absorbing: bool = False, s0: int = 0,
               s1: int | None = None, dtype=np.float64, name: str = "") -> CSRMDP:
    """W x H grid world, 5 actions (N, E, S, W, stay); states [s0, s1)."""
    lib = _load()
    n = W * H
    s1 = n if s1 is None else s1
    m = 5
    goals = grid_goals(W, H, n_goals, seed)
    rows = (s1 - s0) * m
    row_ptr = np.empty(rows + 1, dtype=np.int64)
    nnz = lib.synth_grid_fill(W, H, s0, s1, p_int, p_oth, _ptr(goals), n_goals,
                              1 if absorbing else 0, _ptr(row_ptr), None, None, 0, None, 0)
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=dtype)
    g = np.empty(rows, dtype=dtype)
    is64 = 1 if np.dtype(dtype) == np.float64 else 0
    lib.synth_grid_fill(W, H, s0, s1, p_int, p_oth, _ptr(goals), n_goals, 1 if absorbing else 0,
                        _ptr(row_ptr), _ptr(col), _ptr(val), is64, _ptr(g), is64)
    return CSRMDP(n=n, m=m, gamma=gamma, row_ptr=row_ptr, col=col, val=val, g=g, s0=s0,
                  name=name)


# ---------------------------------------------------------------------------
# Named workloads (the problem shapes the solver is measured on)
# ---------------------------------------------------------------------------

def random_sparse_n1000(dtype=np.float64) -> CSRMDP:
    """n=1000, m=4, 8 successors/row, Dirichlet(1), g~U[0,1], gamma=0.9, seed 1."""
    return random_sparse(1000, 4, 8, 1.0, 0.9, 1, dtype=dtype, name="random_sparse_n1000_m4_k8")


BANDED_4M = dict(n=1 << 22, m=8, k=16, band=4096, alpha=0.5, gamma=0.99, seed=2)


def banded_4m(s0: int = 0, s1: int | None = None, dtype=np.float32, n: int | None = None) -> CSRMDP:
    """n=2^22, m=8, 16 successors/row in a +-4096 band, Dirichlet(0.5), gamma=0.99, seed 2.

    ``n`` overrides the state count (same recipe at a smaller size).
    """
    p = dict(BANDED_4M)
    if n is not None:
        p["n"] = n
    return banded(p["n"], p["m"], p["k"], p["band"], p["alpha"], p["gamma"], p["seed"], s0=s0,
                  s1=s1, dtype=dtype, name=f"banded_n{p['n']}_m8_k16_band4096")


GRID_4096 = dict(W=4096, H=4096, gamma=0.999, seed=3)


def grid_4096(s0: int = 0, s1: int | None = None, dtype=np.float32, side: int | None = None,
              absorbing: bool = False) -> CSRMDP:
    """4096 x 4096 grid world (n = 16.8M), gamma=0.999, 16 goal cells, seed 3."""
    W = H = GRID_4096["W"] if side is None else side
    return grid_world(W, H, GRID_4096["gamma"], GRID_4096["seed"], s0=s0, s1=s1, dtype=dtype,
                      absorbing=absorbing, name=f"grid_{W}x{H}_m5")


def uneven_batch_params(count: int = 512, seed: int = 4, n_lo: float = 2e3, n_hi: float = 2e5):
    """Per-MDP parameters of a batch of independent random MDPs of uneven size.

    n log-uniform in [n_lo, n_hi], m uniform in {2..16}, successors per row
    uniform in {4..32}, gamma uniform in [0.9, 0.999], Dirichlet(1), MDP i
    seeded ``seed*10**6 + i``.
    """
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rs.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(rs.integers(2, 17))
        gamma = float(rs.uniform(0.9, 0.999))
        out.append(dict(n=n, m=m, k_min=4, k_max=32, alpha=1.0, gamma=gamma,
                        seed=seed * 10**6 + i))
    return out


def uneven_mdp(p: dict, dtype=np.float32) -> CSRMDP:
    return random_sparse(p["n"], p["m"], p["k_min"], p["alpha"], p["gamma"], p["seed"],
                         k_max=p["k_max"], dtype=dtype,
                         name=f"random_n{p['n']}_m{p['m']}_k4to32")

"""Building MDPs for the solver from a simulator, from logged transitions or
from PETSc binary files (include/mdp_ingest.h; host-side, no GPU needed).

The madupite paper (section "Implementation") creates an MDP by loading
offline data from earlier experiments or from online simulation, and stores it
in PETSc matrices.  The functions here return a ``HostMDP`` in the layout that
``MDP.from_csr`` takes (row r = s*m + a of an (n*m) x n CSR matrix).  The
arrays are numpy arrays whose memory the library filled through an allocator
callback; with ``pinned=True`` that memory is page-locked (PyTorch's pinned
host allocator), so that ``MDP.from_csr(mdp, host_input=True)`` reads it in
place over the host link.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import capi


@dataclasses.dataclass
class HostMDP:
    """A CSR MDP in host memory: ``row_ptr`` int64[n*m+1], ``col`` int32[nnz],
    ``val`` float64[nnz], ``g`` float64[n*m] (costs, or rewards when
    ``maximize``), discount ``gamma``."""

    n: int
    m: int
    gamma: float
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    g: np.ndarray
    maximize: bool = False

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def rows(self) -> int:
        return self.n * self.m


class _Allocator:
    """The allocator callback: hands the library numpy buffers (page-locked
    ones when pinned) and keeps them by address."""

    def __init__(self, pinned: bool = False):
        if pinned:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("pinned=True needs a CUDA device: page-locked host memory "
                                   "comes from the CUDA driver")
        self.pinned = pinned
        self.bufs = {}
        self.fn = capi.MDP_ALLOC_FN(self._alloc)

    def _alloc(self, nbytes, _user):
        try:
            if self.pinned:
                import torch
                arr = torch.empty(int(nbytes), dtype=torch.uint8, pin_memory=True).numpy()
            else:
                arr = np.empty(int(nbytes), dtype=np.uint8)
            self.bufs[arr.ctypes.data] = arr
            return arr.ctypes.data
        except Exception:  # noqa: BLE001 -- a NULL return is the library's OOM signal
            return None

    def array(self, addr, dtype, count):
        return self.bufs[addr][: count * np.dtype(dtype).itemsize].view(dtype)


def _host_mdp(out, al: _Allocator, gamma, maximize) -> HostMDP:
    n, m, nnz = int(out.n_states), int(out.n_actions), int(out.nnz)
    return HostMDP(n=n, m=m, gamma=float(gamma),
                   row_ptr=al.array(out.row_ptr, np.int64, n * m + 1),
                   col=al.array(out.col, np.int32, nnz), val=al.array(out.val, np.float64, nnz),
                   g=al.array(out.cost, np.float64, n * m), maximize=bool(maximize))


def _int32_cols(c):
    """Successors as int32; one outside int32 becomes -2^31 (reported by the library)."""
    return np.where((c < -2**31) | (c > 2**31 - 1), -2**31, c).astype(np.int32)


def _simulate_states(transitions, cost, s0, s1, m):
    """The raw rows of states [s0, s1): row lengths, successors, probabilities
    and costs in row order (runs in a worker process of from_functions)."""
    rows = (s1 - s0) * m
    lens = np.empty(rows, dtype=np.int64)
    g = np.empty(rows, dtype=np.float64)
    cols, probs = [], []
    r = 0
    for s in range(s0, s1):
        for a in range(m):
            succ, prob = transitions(s, a)
            c = np.asarray(succ, dtype=np.int64).reshape(-1)
            p = np.asarray(prob, dtype=np.float64).reshape(-1)
            if c.shape != p.shape:
                raise ValueError(f"transitions({s}, {a}): {c.size} successors, "
                                 f"{p.size} probabilities")
            lens[r] = c.size
            cols.append(c)
            probs.append(p)
            g[r] = float(cost(s, a))
            r += 1
    empty = np.empty(0, dtype=np.int64)
    return (lens, np.concatenate(cols) if cols else empty,
            np.concatenate(probs) if probs else empty.astype(np.float64), g)


def from_rows(n, m, offsets, col, prob, cost, gamma, threads=0, maximize=False,
              pinned=False) -> HostMDP:
    """Assemble the CSR from raw rows: row r = s*m + a holds the entries
    col/prob[offsets[r]:offsets[r+1]] in any order, repeats allowed (summed);
    cost[r] = g(s, a).  Same result and checks as from_functions."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    col = _int32_cols(np.asarray(col, dtype=np.int64))
    prob = np.ascontiguousarray(prob, dtype=np.float64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    if offsets.shape != (n * m + 1,) or cost.shape != (n * m,):
        raise ValueError("offsets must have n*m+1 entries and cost n*m")
    if col.shape != prob.shape or col.size < int(offsets[-1]):
        raise ValueError("col and prob must hold offsets[-1] entries")
    al = _Allocator(pinned)
    out = capi.mdp_csr_from_rows(n, m, offsets, col, prob, cost, threads=threads, alloc=al.fn)
    return _host_mdp(out, al, gamma, maximize)


def from_functions(n, m, transitions, cost, gamma, threads=1, maximize=False,
                   pinned=False, processes=1) -> HostMDP:
    """Evaluate ``transitions(s, a) -> (successors, probabilities)`` and
    ``cost(s, a) -> float`` for every state-action pair (online simulation).

    Repeated successors are summed and each row is sorted by successor.  With
    threads > 1 the callables are called from several threads (they hold the
    interpreter lock while they run).  With processes > 1 they run in that many
    spawned worker processes over contiguous state ranges instead (they must
    then be picklable: module-level functions), and the rows are assembled by
    the library (from_rows); the result is the same.  An exception raised by a
    callable is re-raised here.
    """
    if processes > 1:
        import multiprocessing as mp
        chunks = max(1, min(n, 4 * processes))
        bounds = [n * i // chunks for i in range(chunks + 1)]
        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.starmap(_simulate_states,
                                 [(transitions, cost, bounds[i], bounds[i + 1], m)
                                  for i in range(chunks)])
        lens = np.concatenate([p[0] for p in parts])
        offsets = np.zeros(n * m + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        return from_rows(n, m, offsets, np.concatenate([p[1] for p in parts]),
                         np.concatenate([p[2] for p in parts]),
                         np.concatenate([p[3] for p in parts]), gamma, threads=threads,
                         maximize=maximize, pinned=pinned)
    errors = []

    def row(s, a, cap, col_p, prob_p, _user):
        try:
            succ, prob = transitions(int(s), int(a))
            c = np.asarray(succ, dtype=np.int64).reshape(-1)
            p = np.asarray(prob, dtype=np.float64).reshape(-1)
            if c.shape != p.shape:
                raise ValueError(f"transitions({s}, {a}): {c.size} successors, "
                                 f"{p.size} probabilities")
            k = c.size
            if 0 < k <= cap:
                np.ctypeslib.as_array(col_p, (k,))[:] = _int32_cols(c)
                np.ctypeslib.as_array(prob_p, (k,))[:] = p
            return k
        except BaseException as e:  # noqa: BLE001 -- carried across the C boundary
            errors.append(e)
            return -1

    def cst(s, a, _user):
        try:
            return float(cost(int(s), int(a)))
        except BaseException as e:  # noqa: BLE001
            errors.append(e)
            return float("nan")

    row_fn, cost_fn = capi.MDP_ROW_FN(row), capi.MDP_COST_FN(cst)
    al = _Allocator(pinned)
    try:
        out = capi.mdp_csr_from_functions(n, m, row_fn, cost_fn, threads=threads, alloc=al.fn)
    except capi.MDPError:
        if errors:
            raise errors[0] from None
        raise
    return _host_mdp(out, al, gamma, maximize)


def from_samples(n, m, s, a, s_next, cost=None, gamma=0.99, unseen="error", unseen_cost=0.0,
                 threads=0, maximize=False, pinned=False) -> HostMDP:
    """The maximum-likelihood MDP of logged transitions (s[i], a[i]) -> s_next[i]
    with cost cost[i]: P(s'|s,a) = N(s,a,s')/N(s,a), g(s,a) = mean cost.
    ``unseen``: "error" or "self_loop" (P(s|s,a) = 1 at ``unseen_cost``) for
    pairs without a sample."""
    s = np.ascontiguousarray(s, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.int32)
    s_next = np.ascontiguousarray(s_next, dtype=np.int64)
    if not (s.shape == a.shape == s_next.shape) or s.ndim != 1:
        raise ValueError("s, a and s_next must be 1-D arrays of one length")
    c = None if cost is None else np.ascontiguousarray(cost, dtype=np.float64)
    if c is not None and c.shape != s.shape:
        raise ValueError("cost must have one entry per sample")
    mode = {"error": capi.MDP_UNSEEN_ERROR, "self_loop": capi.MDP_UNSEEN_SELF_LOOP}[unseen]
    al = _Allocator(pinned)
    out = capi.mdp_csr_from_samples(n, m, s, a, s_next, c, unseen=mode, unseen_cost=unseen_cost,
                                    threads=threads, alloc=al.fn)
    return _host_mdp(out, al, gamma, maximize)


def read_petsc(p_path, g_path=None, gamma=0.99, threads=0, maximize=False,
               pinned=False) -> HostMDP:
    """Load P ((n*m) x n sparse) and g (n x m, dense or sparse) from PETSc
    binary files; g_path None gives zero costs."""
    al = _Allocator(pinned)
    out = capi.mdp_csr_read_petsc(p_path, g_path, threads=threads, alloc=al.fn)
    return _host_mdp(out, al, gamma, maximize)


def write_petsc(mdp, p_path, g_path=None) -> None:
    """Write an object with n, m, row_ptr, col, val, g as PETSc binary files."""
    rp = np.ascontiguousarray(mdp.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(mdp.col, dtype=np.int32)
    val = np.ascontiguousarray(mdp.val, dtype=np.float64)
    g = np.ascontiguousarray(mdp.g, dtype=np.float64)
    if rp.shape != (mdp.n * mdp.m + 1,) or g.shape != (mdp.n * mdp.m,):
        raise ValueError("row_ptr must have n*m+1 entries and g n*m")
    if col.shape != val.shape or col.size < int(rp[-1]):
        raise ValueError("col and val must hold row_ptr[-1] entries")
    c = capi.mdp_host_csr(n_states=mdp.n, n_actions=mdp.m, nnz=int(rp[-1]),
                          row_ptr=rp.ctypes.data, col=col.ctypes.data, val=val.ctypes.data,
                          cost=g.ctypes.data, owned=0)
    capi.mdp_csr_write_petsc(c, p_path, g_path)


def save_npz(mdp, path) -> None:
    """Save an object with n, m, gamma, row_ptr, col, val, g (and optionally
    maximize) as a numpy .npz archive, arrays at their own dtypes."""
    np.savez(path, n=np.int64(mdp.n), m=np.int64(mdp.m), gamma=np.float64(mdp.gamma),
             maximize=np.bool_(getattr(mdp, "maximize", False)),
             row_ptr=np.asarray(mdp.row_ptr), col=np.asarray(mdp.col),
             val=np.asarray(mdp.val), g=np.asarray(mdp.g))


def load_npz(path) -> HostMDP:
    """Load an archive written by save_npz.  The arrays keep their stored dtypes
    (float32 or float64 probabilities and costs); row_ptr becomes int64 and col
    int32.  Shapes are checked here; values are checked by mdp_create."""
    with np.load(path, allow_pickle=False) as z:
        n, m = int(z["n"]), int(z["m"])
        row_ptr = np.ascontiguousarray(z["row_ptr"], dtype=np.int64)
        col = np.ascontiguousarray(z["col"], dtype=np.int32)
        val, g = np.ascontiguousarray(z["val"]), np.ascontiguousarray(z["g"])
        mdp = HostMDP(n=n, m=m, gamma=float(z["gamma"]), row_ptr=row_ptr, col=col, val=val,
                      g=g, maximize=bool(z["maximize"]) if "maximize" in z else False)
    if row_ptr.shape != (n * m + 1,) or g.shape != (n * m,):
        raise ValueError(f"{path}: row_ptr must have n*m+1 entries and g n*m")
    if col.shape != val.shape or col.size != int(row_ptr[-1]):
        raise ValueError(f"{path}: col and val must hold row_ptr[-1] entries")
    if val.dtype not in (np.float32, np.float64) or g.dtype not in (np.float32, np.float64):
        raise ValueError(f"{path}: val and g must be float32 or float64")
    return mdp

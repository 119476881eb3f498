"""Small helpers for tests: build tiny CSR MDPs from dense arrays.

Pure data plumbing (no Bellman arithmetic); used by oracle pins and GPU parity
tests alike.
"""
import numpy as np

from synth import CSRMDP


def from_dense(P, g, gamma, dtype=np.float64, name="dense"):
    """CSR MDP from a dense (n, m, n) transition tensor and (n, m) costs.

    Row s*m + a keeps the nonzero entries of P[s, a] in ascending column order.
    """
    P = np.asarray(P, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    n, m, n2 = P.shape
    assert n == n2 and g.shape == (n, m)
    rows = P.reshape(n * m, n)
    row_ptr = [0]
    col, val = [], []
    for r in range(n * m):
        nz = np.nonzero(rows[r])[0]
        col.extend(nz.tolist())
        val.extend(rows[r, nz].tolist())
        row_ptr.append(len(col))
    return CSRMDP(n=n, m=m, gamma=float(gamma), row_ptr=np.array(row_ptr, dtype=np.int64),
                  col=np.array(col, dtype=np.int32), val=np.array(val, dtype=dtype),
                  g=g.reshape(-1).astype(dtype), name=name)


def random_dense(n, m, rng, density=0.6):
    """Random row-stochastic (n, m, n) tensor with at least one entry per row."""
    P = rng.random((n, m, n)) * (rng.random((n, m, n)) < density)
    for s in range(n):
        for a in range(m):
            if P[s, a].sum() == 0:
                P[s, a, rng.integers(n)] = 1.0
    P /= P.sum(axis=2, keepdims=True)
    return P


def to_dense(mdp):
    """Dense (n, m, n) P and (n, m) g of a whole CSR MDP."""
    n, m = mdp.n, mdp.m
    P = np.zeros((n * m, n))
    for r in range(n * m):
        b, e = mdp.row_ptr[r], mdp.row_ptr[r + 1]
        P[r, mdp.col[b:e]] = mdp.val[b:e]
    return P.reshape(n, m, n), np.asarray(mdp.g, dtype=np.float64).reshape(n, m)

"""Shared helpers of the GPU parity tests (tolerances derived from the arithmetic).

FP32 path: a row sum of k products with non-negative weights summing to 1 has
rounding error at most k*u*max|V| (u = 2^-24, the FP32 unit roundoff; Higham,
"Accuracy and Stability of Numerical Algorithms", 3.1), and g + gamma*sum adds
2u relative.  So |Q_gpu - Q| <= (k + 2) u (max|g| + max|V|); the tests allow
twice that.

Float-float path: products and sums carry ~2^-48 relative error per term
(error-free TwoSum/TwoProd, lower part accumulated in FP32), so the bound is
(k + 6) 2^-48 (max|g| + max|V|); the tests allow 4x that.
"""
import numpy as np
import torch

U32 = 2.0 ** -24
UFF = 2.0 ** -48


def q_tol_f32(mdp, V):
    k = int(np.max(np.diff(mdp.row_ptr)))
    scale = float(np.max(np.abs(mdp.g))) + float(np.max(np.abs(V)))
    return 2.0 * (k + 2) * U32 * scale


def q_tol_ff(mdp, V):
    k = int(np.max(np.diff(mdp.row_ptr)))
    scale = float(np.max(np.abs(mdp.g))) + float(np.max(np.abs(V)))
    return 4.0 * (k + 6) * UFF * scale + 1e-300


def check_greedy(pi_gpu, pi_orc, Q, tol):
    """pi must equal the oracle's wherever the Q-gap exceeds 2*tol; elsewhere the
    GPU's action must attain the minimum within tol (several argmins are valid)."""
    pi_gpu = np.asarray(pi_gpu)
    qmin = Q.min(axis=1)
    q_sorted = np.sort(Q, axis=1)
    gap = (q_sorted[:, 1] - q_sorted[:, 0]) if Q.shape[1] > 1 else np.full(len(Q), np.inf)
    clear = gap > 2 * tol
    assert np.array_equal(pi_gpu[clear], pi_orc[clear]), "greedy action differs on a clear gap"
    qg = Q[np.arange(len(Q)), pi_gpu]
    assert np.all(qg <= qmin + 2 * tol), "greedy action does not attain the minimum"
    assert pi_gpu.min() >= 0 and pi_gpu.max() < Q.shape[1]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()

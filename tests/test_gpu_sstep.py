"""GPU parity of s-step GMRES (blocks of s Krylov vectors orthogonalised together,
the solution update fused into the last block's pass) inside inexact policy
iteration.

* Solves with every block size and restart length reach the oracle's solution:
  dense-LU exact policy iteration for small n, else the oracle's FP64
  certificate ||T V - V||_inf and the bound ||V - V*||_inf <= res / (1 - gamma).
* The Hessenberg matrix an s-step cycle reconstructs matches the FP64 Arnoldi
  matrix of the same Krylov space about as closely as the classical FP32
  Gram-Schmidt cycle does (both orthonormalisations give positive
  subdiagonals, so the bases agree up to rounding), and its least-squares
  record agrees with numpy's solver.
* A residual that is an eigenvector of P (uniform transitions) makes the first
  block exactly dependent: the cycle must end on that breakdown with the exact
  solution (closed form V(s) = g(s) + gamma * mean(g) / (1 - gamma)).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from mdp_helpers import from_dense

pytestmark = pytest.mark.gpu


def _mk(mdp, store="f32"):
    from paper_2502_14474_gb300 import MDP
    return MDP.from_csr(mdp, store=store)


def _certify(mdp, V, pi, tol):
    cert = oracle.certificate(mdp, V)
    assert cert["res_inf"] <= tol * 1.05, cert["res_inf"]
    clear = cert["gap"] > 2 * tol + 1e-12
    assert np.array_equal(pi[clear], cert["pi"][clear])
    return cert


@pytest.mark.parametrize("s_step", [1, 2, 3, 4, 6, 8])
def test_sstep_solve_matches_exact_policy_iteration(s_step):
    mdp = synth.random_sparse_n1000(dtype=np.float32)
    Vs, pis, _, _ = oracle.policy_iteration(mdp)
    h = _mk(mdp)
    tol = 1e-10
    V, pi, st = h.solve(tol=tol, s_step=s_step)
    assert st["converged"]
    Vg, pig = V.cpu().numpy(), pi.cpu().numpy()
    cert = _certify(mdp, Vg, pig, tol)
    assert np.max(np.abs(Vg - Vs)) <= cert["res_inf"] / (1 - mdp.gamma) + 1e-12
    h.close()


@pytest.mark.parametrize("restart", [1, 5, 30, 64])
def test_sstep_restart_lengths(restart):
    """Restart lengths below, equal to and not multiples of the block size."""
    mdp = synth.random_sparse(3000, 4, 8, 1.0, 0.99, seed=120 + restart, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9, restart=restart, s_step=6, max_outer=5000)
    assert st["converged"]
    _certify(mdp, V.cpu().numpy(), pi.cpu().numpy(), 1e-9)
    h.close()


@pytest.mark.parametrize("kind", ["banded", "grid", "random"])
@pytest.mark.parametrize("s_step", [4, 8])
def test_sstep_workload_shapes(kind, s_step):
    """The three workload shapes (banded rows with the shared-memory window,
    short grid rows with the action-major copy, random rows) at sizes spanning
    many tiles and a ragged tail."""
    if kind == "banded":
        mdp = synth.banded(70001, 8, 16, 4096, 0.5, 0.99, seed=131, dtype=np.float32)
    elif kind == "grid":
        mdp = synth.grid_world(181, 173, 0.99, 132, dtype=np.float32)
    else:
        mdp = synth.random_sparse(50003, 5, 12, 1.0, 0.99, seed=133, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9, s_step=s_step)
    assert st["converged"]
    _certify(mdp, V.cpu().numpy(), pi.cpu().numpy(), 1e-9)
    h.close()


@pytest.mark.parametrize("store", ["bf16", "f16"])
def test_sstep_low_precision_inner(store):
    mdp = synth.banded(120000, 8, 16, 3000, 0.5, 0.99, seed=134, dtype=np.float32)
    h = _mk(mdp, store=store)
    V, pi, st = h.solve(tol=1e-9, s_step=6)
    assert st["converged"]
    _certify(mdp, V.cpu().numpy(), pi.cpu().numpy(), 1e-9)
    h.close()


def _one_cycle(mdp, s_step, restart=30):
    from paper_2502_14474_gb300 import capi
    h = _mk(mdp)
    h.solve(tol=0.0, inner_rtol=1e-30, max_outer=1, max_inner=restart, restart=restart,
            s_step=s_step, raise_on_not_converged=False)
    c = capi.mdp_last_cycle(h.h)
    h.close()
    return c


def _exact_first_cycle(mdp, J):
    """FP64 Arnoldi (classical Gram-Schmidt, twice) of the first cycle of a solve
    from V = 0: policy pi_0 = greedy(0), r_0 = T 0 - 0, A = I - gamma P_pi."""
    import scipy.sparse as sp
    TV, pi = oracle.bellman(mdp, np.zeros(mdp.n))
    rows = np.arange(mdp.n) * mdp.m + pi
    b, e = mdp.row_ptr[rows], mdp.row_ptr[rows + 1]
    idx = np.concatenate([np.arange(x, y) for x, y in zip(b, e)])
    P = sp.csr_matrix((mdp.val[idx].astype(np.float64),
                       (np.repeat(np.arange(mdp.n), e - b), mdp.col[idx])), shape=(mdp.n, mdp.n))
    A = sp.eye(mdp.n, format="csr") - mdp.gamma * P
    beta = np.linalg.norm(TV)
    Q = np.zeros((mdp.n, J + 1))
    H = np.zeros((J + 1, J))
    Q[:, 0] = TV / beta
    for j in range(J):
        w = A @ Q[:, j]
        for _ in range(2):
            h = Q[:, :j + 1].T @ w
            w -= Q[:, :j + 1] @ h
            H[:j + 1, j] += h
        H[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / H[j + 1, j]
    return H, beta


def _ls_residuals(H, beta):
    out = []
    for j in range(1, H.shape[1] + 1):
        e = np.zeros(j + 1)
        e[0] = beta
        y = np.linalg.lstsq(H[:j + 1, :j], e, rcond=None)[0]
        out.append(np.linalg.norm(e - H[:j + 1, :j] @ y))
    return np.array(out)


@pytest.mark.parametrize("s_step", [2, 5, 8])
def test_sstep_hessenberg_matches_exact_arnoldi(s_step):
    """Both GPU cycles (classical FP32 Gram-Schmidt and s-step) rebuild the FP64
    Arnoldi matrix of the same Krylov space; the s-step one must be about as
    close to it as the classical one (both keep the basis in FP32)."""
    mdp = synth.banded(40000, 6, 12, 2000, 0.5, 0.99, seed=140, dtype=np.float32)
    Hx, bx = _exact_first_cycle(mdp, 30)
    ref = _one_cycle(mdp, 0)
    c = _one_cycle(mdp, s_step)
    assert ref["J"] == c["J"] == 30
    assert abs(c["beta"] - bx) <= 1e-6 * bx and abs(ref["beta"] - bx) <= 1e-6 * bx
    scale = np.max(np.abs(Hx))
    d_cls = np.max(np.abs(ref["H"] - Hx)) / scale
    d_ss = np.max(np.abs(c["H"] - Hx)) / scale
    print(f"s={s_step} |H_classical - H|/|H| {d_cls:.2e}  |H_sstep - H|/|H| {d_ss:.2e}")
    assert d_ss <= max(20.0 * d_cls, 1e-5)
    rx = _ls_residuals(Hx, bx)
    r_cls = np.max(np.abs(_ls_residuals(ref["H"], ref["beta"]) - rx)) / bx
    r_ss = np.max(np.abs(_ls_residuals(c["H"], c["beta"]) - rx)) / bx
    print(f"  GMRES residuals per step: classical {r_cls:.2e}  s-step {r_ss:.2e} (of beta)")
    # the estimates drive a stop at eta = 0.1 of the outer residual: an error of
    # 1e-4 beta (larger blocks lose digits to the monomial basis' conditioning)
    # cannot change that decision by more than one step
    assert r_ss <= max(20.0 * r_cls, 1e-4)


def test_sstep_least_squares_record():
    mdp = synth.random_sparse(30000, 6, 12, 1.0, 0.99, seed=141, dtype=np.float32)
    c = _one_cycle(mdp, 6)
    J, H, beta, y = c["J"], c["H"], c["beta"], c["y"]
    assert J == 30 and np.all(np.tril(H, -2) == 0.0)
    rhs = np.zeros(J + 1)
    rhs[0] = beta
    y_ref, *_ = np.linalg.lstsq(H, rhs, rcond=None)
    assert np.max(np.abs(y - y_ref)) <= 1e-13 * np.linalg.cond(H) * max(1.0, np.abs(y_ref).max())
    assert abs(c["est"] - np.linalg.norm(rhs - H @ y_ref)) <= 1e-12 * beta


def test_sstep_exact_breakdown_uniform_transitions():
    """One action, uniform transitions: P 1 = 1 and the first residual g is
    mapped by P to the constant mean(g), so the Krylov space of the first cycle
    is span{g, 1} and the block breaks down exactly in its second vector."""
    n, gamma = 400, 0.95
    rng = np.random.default_rng(142)
    g = rng.random((n, 1))
    P = np.full((n, 1, n), 1.0 / n)
    mdp = from_dense(P, g, gamma, dtype=np.float64)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-11, s_step=6)
    assert st["converged"]
    closed = g[:, 0] + gamma * g.mean() / (1 - gamma)
    assert np.max(np.abs(V.cpu().numpy() - closed)) <= 1e-10 / (1 - gamma)
    h.close()


def test_sstep_solves_are_deterministic():
    mdp = synth.banded(60000, 8, 16, 4096, 0.5, 0.99, seed=143, dtype=np.float32)
    h = _mk(mdp)
    V1, pi1, st1 = h.solve(tol=1e-9, s_step=6)
    V2, pi2, st2 = h.solve(tol=1e-9, s_step=6)
    assert torch.equal(V1, V2) and torch.equal(pi1, pi2)
    assert st1["inner_iters"] == st2["inner_iters"]
    h.close()


def test_sstep_rejects_cgs2_and_bad_sizes():
    from paper_2502_14474_gb300 import MDPError, capi
    mdp = synth.random_sparse(500, 2, 4, 1.0, 0.9, seed=144, dtype=np.float32)
    h = _mk(mdp)
    o = capi.mdp_default_opts()
    V = torch.empty(mdp.n, dtype=torch.float64, device="cuda")
    for bad in (-1, 9):
        o.s_step = bad
        with pytest.raises(MDPError):
            capi.mdp_solve(h.h, o, V_out=V)
    o.s_step, o.cgs2 = 4, 1
    with pytest.raises(MDPError):
        capi.mdp_solve(h.h, o, V_out=V)
    h.close()

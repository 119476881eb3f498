"""GPU parity of s-step GMRES (blocks of s Krylov vectors orthogonalised together,
the solution update fused into the last block's pass) inside inexact policy
iteration.

* Solves with every block size and restart length reach the oracle's solution:
  dense-LU exact policy iteration for small n, else the oracle's FP64
  certificate ||T V - V||_inf and the bound ||V - V*||_inf <= res / (1 - gamma).
* The Hessenberg matrix an s-step cycle reconstructs equals the one classical
  Arnoldi builds for the same Krylov space (the basis is the same up to FP32
  rounding: both orthonormalisations give positive subdiagonals), and its
  least-squares record agrees with numpy's solver.
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


@pytest.mark.parametrize("s_step", [2, 5, 8])
def test_sstep_hessenberg_equals_arnoldi(s_step):
    mdp = synth.banded(40000, 6, 12, 2000, 0.5, 0.99, seed=140, dtype=np.float32)
    ref = _one_cycle(mdp, 0)
    c = _one_cycle(mdp, s_step)
    assert ref["J"] == c["J"] == 30
    assert abs(c["beta"] - ref["beta"]) <= 1e-12 * ref["beta"]
    Href, H = ref["H"], c["H"]
    # the basis vectors are FP32 and the two orthogonalisations round
    # differently; the matrices agree to the basis' precision times the
    # conditioning of the block (a few hundred for blocks of up to 8 vectors)
    assert np.max(np.abs(H - Href)) <= 2e-4 * np.max(np.abs(Href))
    # GMRES residual after every step: the same to 1e-4 relative
    for j in range(1, 31):
        e = np.zeros(j + 1)
        e[0] = ref["beta"]
        r_ref = np.linalg.norm(e - Href[:j + 1, :j] @ np.linalg.lstsq(Href[:j + 1, :j], e,
                                                                      rcond=None)[0])
        r = np.linalg.norm(e - H[:j + 1, :j] @ np.linalg.lstsq(H[:j + 1, :j], e, rcond=None)[0])
        assert abs(r - r_ref) <= 1e-4 * ref["beta"]


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

"""GPU tests of BiCGStab (van der Vorst 1992) as the inner solver of inexact
policy iteration: the approximate evaluation step solves (I - gamma P_pi) d = r
with two policy SpMVs per iteration, on the device with no host read between
iterations of a batch.  Results are checked against the FP64 oracle (exact
policy iteration where n is small, the one-sweep certificate elsewhere)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _mdp(kind):
    if kind == "random":
        return synth.random_sparse(3000, 4, 8, 1.0, 0.97, seed=34, dtype=np.float32)
    if kind == "grid":
        return synth.grid_world(48, 40, 0.97, seed=37, dtype=np.float32)
    return synth.banded(40000, 4, 16, 1000, 0.5, 0.97, seed=38, dtype=np.float32)


def _mk(mdp, store="f32"):
    from paper_2502_14474_gb300 import MDP
    return MDP.from_csr(mdp, store=store)


@pytest.mark.parametrize("store", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["random", "grid", "banded"])
def test_bicgstab_solve_meets_the_oracle(store, kind):
    """Every row layout (short rows with the action-major copy, banded rows,
    grid rows); a BF16 handle still runs BiCGStab on its FP32 probabilities."""
    mdp = _mdp(kind)
    h = _mk(mdp, store)
    h.profile(True)
    tol = 1e-9
    V, pi, st = h.solve(tol=tol, inner="bicgstab", max_inner=500)
    k = h.profile_read()["kinds"]["bicgstab_spmv"]
    h.profile(False)
    assert st["converged"]
    assert st["policy_sweeps"] == 2 * st["inner_iters"]
    assert k["launches"] == st["policy_sweeps"]
    Vg = V.cpu().numpy()
    cert = oracle.certificate(mdp, Vg)
    assert cert["res_inf"] <= 1.01 * tol
    clear = cert["gap"] > 1e-8
    assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])
    if kind == "random":
        Vs, _, _, _ = oracle.policy_iteration(mdp)
        assert np.max(np.abs(Vg - Vs)) <= 1.01 * tol / (1 - mdp.gamma)
    h.close()


def test_bicgstab_is_deterministic_and_cheaper_than_sweeps():
    mdp = _mdp("random")
    h = _mk(mdp)
    Va, pa, sa = h.solve(tol=1e-9, inner="bicgstab", max_inner=500)
    Vb, pb, sb = h.solve(tol=1e-9, inner="bicgstab", max_inner=500)
    assert np.array_equal(Va.cpu().numpy(), Vb.cpu().numpy())
    assert np.array_equal(pa.cpu().numpy(), pb.cpu().numpy())
    assert sa["inner_history"] == sb["inner_history"]
    assert sa["residual_history"] == sb["residual_history"]
    # a Krylov solve needs far fewer policy SpMVs than Richardson sweeps at gamma = 0.97
    _, _, sr = h.solve(tol=1e-9, inner="richardson", max_inner=5000)
    assert sa["policy_sweeps"] < sr["policy_sweeps"] / 2
    h.close()


def test_one_bicgstab_iteration_per_outer_step_still_converges():
    """With max_inner = 1 each evaluation is very inexact; the outer loop still
    reaches the tolerance."""
    mdp = synth.random_sparse(800, 3, 6, 1.0, 0.9, seed=35, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9, inner="bicgstab", max_inner=1, max_outer=2000)
    assert st["converged"] and max(st["inner_history"]) <= 1
    Vs, _, _, _ = oracle.policy_iteration(mdp)
    assert np.max(np.abs(V.cpu().numpy() - Vs)) <= 1.01e-9 / (1 - mdp.gamma)
    h.close()

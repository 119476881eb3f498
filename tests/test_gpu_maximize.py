"""GPU tests of reward maximisation (MDP_FLAG_MAXIMIZE).

Maximising rewards r is minimising costs g = -r with V_max = -V_min and the
same policy: max_a [r + gamma P V] = -min_a [-r + gamma P (-V)], and the lowest
maximising action is the lowest minimising one.  IEEE round-to-nearest is
symmetric under negation, so a maximising handle must return bitwise the
negated outputs of a minimising handle given -r and -V.  The oracle (a
minimiser) checks the values through that identity.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev, q_tol_f32, q_tol_ff

pytestmark = pytest.mark.gpu


def _pair(store="f32", seed=31, n=3000, m=5):
    from paper_2502_14474_gb300 import MDP
    base = synth.random_sparse(n, m, 12, 1.0, 0.95, seed=seed, dtype=np.float32)
    rewards = base.g.copy()                       # r(s, a) ~ U[0, 1]
    as_cost = dataclasses.replace(base, g=-rewards)
    hmax = MDP.from_csr(base, store=store, maximize=True)
    hmin = MDP.from_csr(as_cost, store=store)
    return base, as_cost, hmax, hmin


def _same_neg(a, b):
    """a == -b elementwise (exact; signed zeros compare equal)."""
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.array_equal(a, -b)


@pytest.mark.parametrize("vt", [torch.float32, torch.float64])
def test_bellman_is_negated_minimisation(vt):
    base, as_cost, hmax, hmin = _pair()
    assert hmax.info()["maximize"] == 1 and hmin.info()["maximize"] == 0
    V = torch.from_numpy(np.random.default_rng(2).uniform(0, 20, base.n)).to("cuda", vt)
    a = hmax.bellman(V, want_r=True)
    b = hmin.bellman(-V, want_r=True)
    assert _same_neg(a["V"], b["V"]) and _same_neg(a["r"], b["r"])
    assert torch.equal(a["pi"], b["pi"])
    assert a["res_inf"] == b["res_inf"] and a["res_2"] == b["res_2"]
    # the definition, through the oracle's minimiser on the costs -r
    Vn = -V.double().cpu().numpy()
    TVmin, pimin = oracle.bellman(as_cost, Vn)
    tol = q_tol_ff(as_cost, Vn) if vt == torch.float64 else q_tol_f32(as_cost, Vn)
    assert np.max(np.abs(a["V"].double().cpu().numpy() + TVmin)) <= tol
    hmax.close(), hmin.close()


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_solve_is_negated_minimisation(store):
    base, as_cost, hmax, hmin = _pair(store=store, seed=32)
    tol = 1e-9
    Va, pia, sa = hmax.solve(tol=tol)
    Vb, pib, sb = hmin.solve(tol=tol)
    assert _same_neg(Va, Vb) and torch.equal(pia, pib)
    for k in ("outer_iters", "inner_iters", "bellman_sweeps", "policy_sweeps", "residual_inf",
              "residual_history", "inner_history"):
        assert sa[k] == sb[k], k
    # V_max is the reward-maximising fixed point: -V* of the cost problem
    Vs, pis, _, _ = oracle.policy_iteration(as_cost)
    assert sa["converged"]
    assert np.max(np.abs(Va.cpu().numpy() + Vs)) <= 1.05 * tol / (1 - base.gamma)
    cert = oracle.certificate(as_cost, -Va.cpu().numpy())
    assert cert["res_inf"] <= 1.05 * tol
    clear = cert["gap"] > 1e-8
    assert np.array_equal(pia.cpu().numpy()[clear], pis[clear])
    hmax.close(), hmin.close()


def test_warm_start_and_policy_eval_are_negated():
    base, as_cost, hmax, hmin = _pair(seed=33)
    rng = np.random.default_rng(3)
    V0 = torch.from_numpy(rng.uniform(0, 20, base.n)).to("cuda")
    Va, pia, sa = hmax.solve(tol=1e-8, V_init=V0)
    Vb, pib, sb = hmin.solve(tol=1e-8, V_init=-V0)
    assert _same_neg(Va, Vb) and torch.equal(pia, pib) and sa["inner_iters"] == sb["inner_iters"]
    pi = dev(rng.integers(0, base.m, size=base.n).astype(np.int32))
    va, vb = V0.clone(), -V0
    ea = hmax.policy_eval(pi, va, 1e-9)
    eb = hmin.policy_eval(pi, vb, 1e-9)
    assert _same_neg(va, vb) and ea == eb
    # v_pi of the rewards: -v_pi of the costs -r
    Vpi = oracle.policy_evaluate(as_cost, pi.cpu().numpy())
    assert np.max(np.abs(va.cpu().numpy() + Vpi)) <= 1.01e-9 / (1 - base.gamma) + 1e-13
    hmax.close(), hmin.close()

"""GPU solves of MDPs built by the host ingest paths (include/mdp_ingest.h):
a PETSc file read into page-locked memory and created in place, the
maximum-likelihood model of logged samples, and a simulator's callbacks.
Each solve is checked against the FP64 oracle on the same CSR."""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _as_oracle(h):
    return synth.CSRMDP(n=h.n, m=h.m, gamma=h.gamma, row_ptr=h.row_ptr, col=h.col, val=h.val,
                        g=h.g)


def _check_solution(h, V, pi, st, tol):
    ref = _as_oracle(h)
    Vg = V.cpu().numpy()
    cert = oracle.certificate(ref, Vg)
    assert st["converged"] and cert["res_inf"] <= 1.05 * tol
    clear = cert["gap"] > 1e-8
    assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])


def test_petsc_file_pinned_in_place_create(tmp_path):
    from paper_2502_14474_gb300 import MDP, ingest
    mdp = synth.banded(20000, 4, 8, 256, 0.5, 0.99, seed=9, dtype=np.float32)
    p, g = os.path.join(tmp_path, "P.bin"), os.path.join(tmp_path, "g.bin")
    ingest.write_petsc(mdp, p, g)
    hm = ingest.read_petsc(p, g, gamma=mdp.gamma, pinned=True)
    x = torch.from_numpy(hm.val)
    assert x.is_pinned()
    tol = 1e-9
    with MDP.from_csr(hm, host_input=True) as h1, MDP.from_csr(hm) as h2:
        V1, pi1, st1 = h1.solve(tol=tol)
        V2, pi2, st2 = h2.solve(tol=tol)
        torch.cuda.synchronize()
    # the in-place (page-locked) and the device-copy creates hold the same matrix
    assert torch.equal(V1, V2) and torch.equal(pi1, pi2)
    assert st1["inner_iters"] == st2["inner_iters"]
    _check_solution(hm, V1, pi1, st1, tol)


@pytest.mark.parametrize("maximize", [False, True])
def test_solve_of_the_sample_model(maximize):
    from paper_2502_14474_gb300 import MDP, ingest
    truth = synth.random_sparse(500, 3, 6, 1.0, 0.95, seed=41, dtype=np.float64)
    rng = np.random.default_rng(5)
    per = 40  # samples per state-action pair
    rows = truth.n * truth.m
    r = np.repeat(np.arange(rows), per)
    # successor of each sample drawn by inverse CDF within its row
    cdf = np.cumsum(truth.val)
    u = rng.random(r.size)
    lo = truth.row_ptr[r]
    base = np.where(lo > 0, cdf[np.maximum(lo - 1, 0)], 0.0)
    span = cdf[truth.row_ptr[r + 1] - 1] - base
    idx = np.searchsorted(cdf, base + u * span, side="right")
    idx = np.minimum(idx, truth.row_ptr[r + 1] - 1)
    s_next = truth.col[idx]
    costs = truth.g[r] + 0.1 * rng.normal(size=r.size)
    hm = ingest.from_samples(truth.n, truth.m, r // truth.m, r % truth.m, s_next, costs,
                             gamma=truth.gamma, maximize=maximize)
    assert hm.nnz <= truth.nnz and np.all(np.isin(hm.col, truth.col))
    tol = 1e-9
    with MDP.from_csr(hm) as h:
        V, pi, st = h.solve(tol=tol)
    if maximize:  # rewards: the solution is -V of the costs -g
        neg = _as_oracle(hm)
        neg.g = -hm.g
        cert = oracle.certificate(neg, -V.cpu().numpy())
        assert st["converged"] and cert["res_inf"] <= 1.05 * tol
        clear = cert["gap"] > 1e-8
        assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])
    else:
        _check_solution(hm, V, pi, st, tol)


def test_solve_of_a_simulator():
    from paper_2502_14474_gb300 import MDP, ingest
    W = 40  # a W x W grid; actions N/E/S/W; slip to a random neighbour with p = 0.2
    moves = [(0, 1), (1, 0), (0, -1), (-1, 0)]

    def cell(x, y):
        return min(max(y, 0), W - 1) * W + min(max(x, 0), W - 1)

    def transitions(s, a):
        x, y = s % W, s // W
        succ = [cell(x + dx, y + dy) for dx, dy in moves]
        prob = [0.05] * 4
        prob[a] += 0.8
        return succ + [s], prob + [0.0]

    def cost(s, a):
        return 0.0 if s == W * W - 1 else 1.0
    hm = ingest.from_functions(W * W, 4, transitions, cost, gamma=0.98, threads=4)
    tol = 1e-9
    with MDP.from_csr(hm) as h:
        V, pi, st = h.solve(tol=tol)
    _check_solution(hm, V, pi, st, tol)
    Vs, _, _, _ = oracle.policy_iteration(_as_oracle(hm))
    assert np.max(np.abs(V.cpu().numpy() - Vs)) <= 1.05 * tol / (1 - hm.gamma)

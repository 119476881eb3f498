"""The FP32-screened float-float Bellman backup against the full float-float pass.

The screened kernel sums every row in FP32 over the high parts of V, keeps
only the actions whose rounding-error interval reaches the state's smallest
upper bound, and repeats those rows in float-float with the same operations
as the full pass.  Its outputs must therefore be bitwise those of the full
pass (the default; environment MDP_FF_SCREEN at create selects the screen):
V' = T V, the greedy policy (lowest minimising action), the residual
r = T V - V and both residual norms, on random value vectors, on the fixed
point (where action gaps are smallest relative to V), and on rows built to
tie exactly or within one ulp.  The oracle's FP64 backup certifies the shared
result.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _pair(mdp, monkeypatch):
    from paper_2502_14474_gb300 import MDP
    monkeypatch.setenv("MDP_FF_SCREEN", "1")
    hs = MDP.from_csr(mdp)
    monkeypatch.delenv("MDP_FF_SCREEN")
    hf = MDP.from_csr(mdp)
    assert hs.info()["ff_screen"] == 1 and hs.info()["window"] == 1
    assert hf.info()["ff_screen"] == 0
    return hs, hf


def _same(hs, hf, V):
    a = hs.bellman(V, want_r=True)
    b = hf.bellman(V, want_r=True)
    assert torch.equal(a["V"], b["V"])
    assert torch.equal(a["pi"], b["pi"])
    assert torch.equal(a["r"], b["r"])
    assert a["res_inf"] == b["res_inf"] and a["res_2"] == b["res_2"]
    return a


def _check_oracle(mdp, V, out):
    TV, pi = oracle.bellman(mdp, V.cpu().numpy())
    Vg = out["V"].cpu().numpy()
    scale = np.max(np.abs(TV))
    assert np.max(np.abs(Vg - TV)) <= 1e-12 * scale
    cert = oracle.certificate(mdp, V.cpu().numpy())
    clear = cert["gap"] > 1e-10 * scale
    assert np.array_equal(out["pi"].cpu().numpy()[clear], pi[clear])


@pytest.mark.parametrize("m", [2, 4, 8, 16, 32])
def test_screen_bitwise_random_values(m, monkeypatch):
    """Rows of 16 aligned entries (4 lanes a row), 2 to 32 actions; a ragged
    last tile (n not a multiple of the tile)."""
    k = 16
    mdp = synth.banded(40003, m, k, 600, 0.5, 0.99, seed=300 + m + k, dtype=np.float32)
    hs, hf = _pair(mdp, monkeypatch)
    rng = np.random.default_rng(301)
    for scale in (1.0, 100.0):
        V = torch.from_numpy(scale * rng.random(mdp.n)).cuda()
        out = _same(hs, hf, V)
        _check_oracle(mdp, V, out)
    hs.close()
    hf.close()


def test_screen_bitwise_at_the_fixed_point(monkeypatch):
    """Near V*, the greedy gaps are what they are at convergence; the backup at
    V* returns V* itself up to the tolerance."""
    mdp = synth.banded(60000, 8, 16, 1000, 0.5, 0.99, seed=302, dtype=np.float32)
    hs, hf = _pair(mdp, monkeypatch)
    V, pi, st = hs.solve(tol=1e-10)
    out = _same(hs, hf, V)
    assert out["res_inf"] <= 1.05e-10
    assert torch.equal(out["pi"], pi)
    _check_oracle(mdp, V, out)
    hs.close()
    hf.close()


def _with_ties(mdp):
    """Copy row (s, 0) into (s, 3) with the same cost (an exact tie, which the
    lowest action wins), into (s, 5) with the cost one ulp lower (a winner
    inside the screening interval of the others) and into (s, 6) with its
    entries reversed and the cost one ulp higher (a float-float sum of other
    rounding, inside the interval too)."""
    m, k = mdp.m, mdp.row_ptr[1] - mdp.row_ptr[0]
    col = mdp.col.reshape(mdp.n, m, k).copy()
    val = mdp.val.reshape(mdp.n, m, k).copy()
    g = mdp.g.reshape(mdp.n, m).copy()
    col[:, 3], val[:, 3], g[:, 3] = col[:, 0], val[:, 0], g[:, 0]
    col[:, 5], val[:, 5] = col[:, 0], val[:, 0]
    g[:, 5] = np.nextafter(g[:, 0], np.float32(-np.inf))
    col[:, 6], val[:, 6] = col[:, 0, ::-1], val[:, 0, ::-1]
    g[:, 6] = np.nextafter(g[:, 0], np.float32(np.inf))
    return synth.CSRMDP(n=mdp.n, m=m, gamma=mdp.gamma, row_ptr=mdp.row_ptr, col=col.ravel(),
                        val=val.ravel(), g=g.ravel())


def test_screen_bitwise_on_near_ties(monkeypatch):
    base = synth.banded(50001, 8, 16, 800, 0.5, 0.99, seed=303, dtype=np.float32)
    mdp = _with_ties(base)
    hs, hf = _pair(mdp, monkeypatch)
    rng = np.random.default_rng(304)
    V = torch.from_numpy(10.0 * rng.random(mdp.n)).cuda()
    out = _same(hs, hf, V)
    pi = out["pi"].cpu().numpy()
    TV, pi_o, Q, _ = oracle.bellman(mdp, V.cpu().numpy(), want_q=True)
    scale = np.max(np.abs(TV))
    assert np.max(np.abs(out["V"].cpu().numpy() - TV)) <= 1e-12 * scale
    # action 3 ties action 0 exactly and action 6 is never below it: neither wins
    assert not np.any(pi == 3) and not np.any(pi == 6)
    others = np.min(Q[:, [1, 2, 4, 7]], axis=1)
    g0 = mdp.g.reshape(mdp.n, 8)[:, 0]
    # the family wins clearly and its one-ulp split is resolvable in float-float
    fam = (Q[:, 5] < others - 1e-9 * scale) & (g0 >= 2.0 ** -10)
    assert np.count_nonzero(fam) > 1000
    assert np.all(pi[fam] == 5)
    clear = others < Q[:, 5] - 1e-9 * scale
    assert np.array_equal(pi[clear], pi_o[clear])
    hs.close()
    hf.close()


def test_screen_full_solves_are_bitwise_equal(monkeypatch):
    """Every backup of the solve is bitwise equal, so the whole solve is."""
    mdp = synth.banded(80000, 8, 16, 2000, 0.5, 0.99, seed=305, dtype=np.float32)
    hs, hf = _pair(mdp, monkeypatch)
    V1, pi1, st1 = hs.solve(tol=1e-9)
    V2, pi2, st2 = hf.solve(tol=1e-9)
    assert torch.equal(V1, V2) and torch.equal(pi1, pi2)
    assert st1["outer_iters"] == st2["outer_iters"]
    assert st1["inner_iters"] == st2["inner_iters"]
    cert = oracle.certificate(mdp, V1.cpu().numpy())
    assert cert["res_inf"] <= 1.05e-9
    hs.close()
    hf.close()


def test_screen_off_where_it_does_not_apply(monkeypatch):
    """Five actions (not a power of two), a band too wide for the ring, rows of
    12 or of 8 entries (not read by the 16-entry fast path): the full pass runs."""
    from paper_2502_14474_gb300 import MDP
    monkeypatch.setenv("MDP_FF_SCREEN", "1")
    for mdp in (synth.banded(40000, 5, 16, 600, 0.5, 0.99, seed=306, dtype=np.float32),
                synth.random_sparse(40000, 8, 16, 1.0, 0.99, seed=307, dtype=np.float32),
                synth.banded(30000, 8, 12, 600, 0.5, 0.99, seed=308, dtype=np.float32),
                synth.banded(30000, 4, 8, 600, 0.5, 0.99, seed=309, dtype=np.float32)):
        h = MDP.from_csr(mdp)
        assert h.info()["ff_screen"] == 0
        h.close()

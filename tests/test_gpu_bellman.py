"""GPU parity of the fused Bellman backup (K1 FP32, K6 float-float) vs the oracle.

Each case runs mdp_bellman through the C ABI and compares T V, the greedy
policy and the residual norms with the FP64 oracle on the same seeded input.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import check_greedy, dev, q_tol_f32, q_tol_ff
from mdp_helpers import from_dense, random_dense

pytestmark = pytest.mark.gpu


def _mk(mdp, store="f32"):
    from paper_2502_14474_gb300 import MDP
    return MDP.from_csr(mdp, store=store)


def _compare(mdp, V, path):
    """Run one backup on the GPU and check it against the oracle."""
    h = _mk(mdp)
    if path == "f32":
        Vt = dev(V.astype(np.float32))
        Vd = V.astype(np.float32).astype(np.float64)
        tol = q_tol_f32(mdp, Vd)
    else:
        Vt = dev(V.astype(np.float64))
        Vd = V.astype(np.float64)
        tol = q_tol_ff(mdp, Vd)
    out = h.bellman(Vt, want_r=True)
    TV, pi, Q, _ = oracle.bellman(mdp, Vd, want_q=True)
    TVg = out["V"].double().cpu().numpy()
    assert np.max(np.abs(TVg - TV)) <= tol, (np.max(np.abs(TVg - TV)), tol)
    check_greedy(out["pi"].cpu().numpy(), pi, Q, tol)
    r = TV - Vd
    rtol_abs = tol + 2.0 ** -24 * np.max(np.abs(r))  # r is stored in FP32
    assert np.max(np.abs(out["r"].double().cpu().numpy() - r)) <= rtol_abs + tol
    assert abs(out["res_inf"] - np.max(np.abs(r))) <= rtol_abs + tol
    assert abs(out["res_2"] - np.linalg.norm(r)) <= (rtol_abs + tol) * np.sqrt(mdp.n)
    h.close()
    return out


@pytest.mark.parametrize("path", ["f32", "ff"])
def test_random_sparse_n1000(path):
    mdp = synth.random_sparse_n1000()
    V = np.random.default_rng(1).random(mdp.n) * 5
    _compare(mdp, V, path)


@pytest.mark.parametrize("path", ["f32", "ff"])
@pytest.mark.parametrize("n,m,kmin,kmax", [(1, 1, 1, 1), (7, 1, 3, 3), (300, 16, 1, 1),
                                           (513, 3, 33, 33), (1000, 5, 1, 40),
                                           (2049, 2, 12, 20), (129, 64, 2, 9)])
def test_odd_shapes(path, n, m, kmin, kmax):
    k = min(kmin, n)
    mdp = synth.random_sparse(n, m, k, 1.0, 0.95, seed=n * 7 + m, k_max=min(kmax, n),
                              dtype=np.float32)
    V = np.random.default_rng(n).normal(size=n) * 10
    _compare(mdp, V, path)


@pytest.mark.parametrize("path", ["f32", "ff"])
def test_banded_small_edges(path):
    # band clipped at both matrix edges, tiles straddle the ends
    mdp = synth.banded(10007, 8, 16, 4096, 0.5, 0.99, seed=2, dtype=np.float32)
    V = np.random.default_rng(3).random(mdp.n) * 100
    _compare(mdp, V, path)


@pytest.mark.parametrize("path", ["f32", "ff"])
def test_grid_world_small(path):
    mdp = synth.grid_world(37, 29, 0.999, seed=3, dtype=np.float32)
    V = np.random.default_rng(4).random(mdp.n) * 1000
    _compare(mdp, V, path)


@pytest.mark.parametrize("path", ["f32", "ff"])
def test_many_actions(path):
    """Short Q tiles: 40 actions on random rows (tiles of a few states, no
    window) and 100 actions on banded rows (the shared-memory window with its
    largest Q tile)."""
    rng = np.random.default_rng(12)
    for mdp in (synth.random_sparse(3001, 40, 6, 1.0, 0.95, seed=13, dtype=np.float32),
                synth.banded(40000, 100, 16, 200, 0.5, 0.99, seed=14, dtype=np.float32)):
        V = rng.random(mdp.n) * 20
        _compare(mdp, V, path)


def test_ties_take_lowest_action():
    rng = np.random.default_rng(5)
    n, m = 300, 6
    P1 = random_dense(n, 1, rng, density=0.05)
    P = np.repeat(P1, m, axis=1)
    g = np.repeat(rng.random((n, 1)), m, axis=1)
    mdp = from_dense(P, g, 0.9, dtype=np.float32)
    from paper_2502_14474_gb300 import MDP
    h = MDP.from_csr(mdp)
    for dt in (torch.float32, torch.float64):
        out = h.bellman(torch.rand(n, dtype=dt, device="cuda"))
        assert int(out["pi"].max()) == 0
    h.close()


def test_f64_inputs_keep_full_precision():
    # FP64 probabilities and costs: the float-float path keeps the low parts
    mdp = synth.random_sparse(2000, 4, 8, 1.0, 0.9, seed=9, dtype=np.float64)
    V = np.random.default_rng(6).random(mdp.n) * 10
    out = _compare(mdp, V, "ff")
    TV, _ = oracle.bellman(mdp, V)
    err = np.max(np.abs(out["V"].cpu().numpy() - TV))
    assert err <= 1e-11, err


def test_zero_value_vector_gives_costs():
    mdp = synth.random_sparse(500, 3, 5, 1.0, 0.9, seed=10, dtype=np.float32)
    from paper_2502_14474_gb300 import MDP
    h = MDP.from_csr(mdp)
    out = h.bellman(torch.zeros(mdp.n, dtype=torch.float64, device="cuda"))
    g = mdp.g.reshape(mdp.n, mdp.m).astype(np.float64)
    assert np.array_equal(out["V"].cpu().numpy(), g.min(axis=1))
    assert np.array_equal(out["pi"].cpu().numpy(), np.argmin(g, axis=1))
    h.close()


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("where", ["pageable", "pinned", "pinned_staged"])
@pytest.mark.parametrize("f64", [False, True])
def test_host_input_matches_device_input(where, f64, monkeypatch):
    """Host inputs are staged on the device (pageable memory) or read in place by
    the packing kernel (page-locked memory); both give the device-input handle."""
    mdp = synth.random_sparse(3000, 4, 10, 1.0, 0.95, seed=11,
                              dtype=np.float64 if f64 else np.float32)
    from paper_2502_14474_gb300 import MDP
    a = MDP.from_csr(mdp)
    arrs = [mdp.row_ptr, mdp.col, mdp.val, mdp.g]
    if where != "pageable":
        arrs = [_pinned(x) for x in arrs]
    if where == "pinned_staged":
        monkeypatch.setenv("MDP_STAGE_HOST_INPUT", "1")
    b = MDP(mdp.n, mdp.m, *arrs, mdp.gamma)
    monkeypatch.delenv("MDP_STAGE_HOST_INPUT", raising=False)
    V = torch.rand(mdp.n, dtype=torch.float64, device="cuda")
    oa, ob = a.bellman(V), b.bellman(V)
    assert torch.equal(oa["V"], ob["V"]) and torch.equal(oa["pi"], ob["pi"])
    assert oa["res_inf"] == ob["res_inf"] and oa["res_2"] == ob["res_2"]
    assert a.info() == b.info()
    a.close()
    b.close()


def test_deterministic_reductions():
    mdp = synth.banded(50000, 4, 8, 500, 0.5, 0.99, seed=12, dtype=np.float32)
    from paper_2502_14474_gb300 import MDP
    h = MDP.from_csr(mdp)
    V = torch.rand(mdp.n, dtype=torch.float64, device="cuda") * 50
    outs = [h.bellman(V, want_r=True) for _ in range(3)]
    for o in outs[1:]:
        assert o["res_2"] == outs[0]["res_2"] and o["res_inf"] == outs[0]["res_inf"]
        assert torch.equal(o["r"], outs[0]["r"])
    h.close()


@pytest.mark.parametrize("where", ["device", "pinned"])
@pytest.mark.parametrize("bad", ["not_stochastic", "nan", "col_range", "empty_row", "neg",
                                 "gamma", "rowptr"])
def test_create_rejects_bad_input(bad, where):
    from paper_2502_14474_gb300 import MDP, MDPError
    mdp = synth.random_sparse(100, 2, 4, 1.0, 0.9, seed=13, dtype=np.float32)
    val, col, rp, g, gamma = mdp.val.copy(), mdp.col.copy(), mdp.row_ptr.copy(), mdp.g.copy(), 0.9
    expect = {"not_stochastic": "MDP_ERR_NOT_STOCHASTIC", "nan": "MDP_ERR_NONFINITE",
              "col_range": "MDP_ERR_BAD_CSR", "empty_row": "MDP_ERR_NOT_STOCHASTIC",
              "neg": "MDP_ERR_NOT_STOCHASTIC", "gamma": "MDP_ERR_ARG",
              "rowptr": "MDP_ERR_BAD_CSR"}[bad]
    if bad == "not_stochastic":
        val[5] *= 1.5
    elif bad == "nan":
        g[7] = np.nan
    elif bad == "col_range":
        col[11] = 100
    elif bad == "empty_row":
        rp[3:] -= 0
        rp[3] = rp[2]  # row 2 empty, row 3 twice as long: not stochastic
    elif bad == "neg":
        val[2] = -val[2]
    elif bad == "gamma":
        gamma = 1.0
    elif bad == "rowptr":
        rp[10] = rp[11] + 1
    put = dev if where == "device" else _pinned
    with pytest.raises(MDPError) as ei:
        MDP(mdp.n, mdp.m, put(rp), put(col), put(val), put(g), gamma)
    assert ei.value.status_name == expect


def test_bad_arguments_are_errors_not_faults():
    from paper_2502_14474_gb300 import MDP, MDPError, capi
    mdp = synth.random_sparse(100, 2, 4, 1.0, 0.9, seed=14, dtype=np.float32)
    h = MDP.from_csr(mdp)
    V = torch.zeros(mdp.n, device="cuda")
    with pytest.raises(MDPError):
        capi.mdp_bellman(h.h, V, 7)  # bad dtype
    with pytest.raises(MDPError):
        capi.mdp_bellman(h.h, V, capi.MDP_F32, V_out=V)  # aliasing
    bad_pi = torch.full((mdp.n,), 5, dtype=torch.int32, device="cuda")
    with pytest.raises(MDPError):
        h.policy_eval(bad_pi, torch.zeros(mdp.n, dtype=torch.float64, device="cuda"), 1e-6)
    with pytest.raises(MDPError):
        capi.mdp_create(0, 1, 0, 0, 0, 0, 0, 0, 0.5, 0)
    h.close()


def test_banded_4m_full_size_sampled(banded_4m_gpu):
    """Full-size banded workload (n = 2^22, m = 8, 16 nnz/row): FP32 and float-float
    backups checked state by state on sampled blocks (both edges and the middle)."""
    mdp, h = banded_4m_gpu
    n = mdp.n
    rng = np.random.default_rng(15)
    V = rng.random(n) * 100
    for path in ("f32", "ff"):
        Vt = dev(V.astype(np.float32)) if path == "f32" else dev(V)
        Vd = V.astype(np.float32).astype(np.float64) if path == "f32" else V
        out = h.bellman(Vt, want_r=True)
        TVg = out["V"].double().cpu().numpy()
        pig = out["pi"].cpu().numpy()
        tol = q_tol_f32(mdp, Vd) if path == "f32" else q_tol_ff(mdp, Vd)
        for s0 in (0, n // 2 - 1000, n - 3000):
            s1 = s0 + 3000
            blk = synth.banded_4m(s0=s0, s1=s1)
            TV, pi, Q, _ = oracle.bellman(blk, Vd, want_q=True)
            assert np.max(np.abs(TVg[s0:s1] - TV)) <= tol
            check_greedy(pig[s0:s1], pi, Q, tol)
        # residual norm against its definition on the whole vector (r is FP32)
        r = TVg - Vd
        assert abs(out["res_inf"] - np.max(np.abs(r))) <= 2 * tol + 2.0 ** -24 * np.max(np.abs(r))


@pytest.mark.parametrize("path", ["f32", "ff"])
@pytest.mark.parametrize("n,m,k,band", [(200003, 8, 16, 1000), (120000, 5, 5, 3000),
                                        (70001, 3, 7, 2000)])
def test_window_kernel_matches_global_gathers(path, n, m, k, band, monkeypatch):
    """The banded kernel that stages V in a shared-memory ring gives bitwise the
    same T V, pi and r as the global-gather kernel (same per-row summation order)
    and matches the oracle."""
    from paper_2502_14474_gb300 import MDP
    mdp = synth.banded(n, m, k, band, 0.5, 0.99, seed=n % 97, dtype=np.float32)
    V = np.random.default_rng(7).random(n) * 50
    Vt = dev(V.astype(np.float32)) if path == "f32" else dev(V)
    win = MDP.from_csr(mdp)
    monkeypatch.setenv("MDP_NO_WINDOW", "1")
    glob = MDP.from_csr(mdp)
    monkeypatch.delenv("MDP_NO_WINDOW")
    a = win.bellman(Vt, want_r=True)
    b = glob.bellman(Vt, want_r=True)
    assert torch.equal(a["V"], b["V"]) and torch.equal(a["pi"], b["pi"])
    assert torch.equal(a["r"], b["r"]) and a["res_inf"] == b["res_inf"]
    assert abs(a["res_2"] - b["res_2"]) <= 1e-12 * b["res_2"]
    Vd = V.astype(np.float32).astype(np.float64) if path == "f32" else V
    tol = q_tol_f32(mdp, Vd) if path == "f32" else q_tol_ff(mdp, Vd)
    TV, pi, Q, _ = oracle.bellman(mdp, Vd, want_q=True)
    assert np.max(np.abs(a["V"].double().cpu().numpy() - TV)) <= tol
    check_greedy(a["pi"].cpu().numpy(), pi, Q, tol)
    win.close()
    glob.close()

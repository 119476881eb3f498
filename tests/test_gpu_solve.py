"""GPU parity of policy evaluation (GMRES) and inexact policy iteration.

Policy evaluation is checked against the oracle's dense-LU solve of
(I - gamma P_pi) v = g_pi, and against the oracle's T_pi through the residual.
mdp_solve is checked against exact policy iteration (dense LU) where n is
small, and otherwise through the oracle's FP64 certificate ||T V - V||_inf
and the bound ||V - V*||_inf <= ||T V - V||_inf / (1 - gamma).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _mk(mdp, store="f32"):
    from paper_2502_14474_gb300 import MDP
    return MDP.from_csr(mdp, store=store)


def _policy_residual_2(mdp, pi, v):
    return float(np.linalg.norm(oracle.policy_apply(mdp, pi, v) - v))


# ---------------------------------------------------------------- policy eval

@pytest.mark.parametrize("restart", [1, 5, 30, 64])
def test_policy_eval_matches_dense_solve(restart):
    mdp = synth.random_sparse_n1000()
    pi = np.random.default_rng(restart).integers(0, mdp.m, size=mdp.n).astype(np.int32)
    Vpi = oracle.policy_evaluate(mdp, pi)
    h = _mk(mdp)
    v = torch.zeros(mdp.n, dtype=torch.float64, device="cuda")
    tol = 1e-10
    st = h.policy_eval(dev(pi), v, tol, restart=restart, max_iters=20000)
    vg = v.cpu().numpy()
    assert st["converged"]
    # ||v - V_pi||_inf <= ||(I - gamma P)^-1||_inf ||res||_inf <= ||res||_2 / (1 - gamma)
    assert np.max(np.abs(vg - Vpi)) <= 1.01 * tol / (1 - mdp.gamma) + 1e-13
    assert _policy_residual_2(mdp, pi, vg) <= 1.01 * tol + 1e-13
    h.close()


def test_policy_eval_f32_vector_and_warm_start():
    mdp = synth.random_sparse(3000, 5, 12, 1.0, 0.95, seed=21, dtype=np.float32)
    pi = np.random.default_rng(1).integers(0, mdp.m, size=mdp.n).astype(np.int32)
    Vpi = oracle.policy_evaluate(mdp, pi)
    h = _mk(mdp)
    v = torch.zeros(mdp.n, dtype=torch.float32, device="cuda")
    st = h.policy_eval(dev(pi), v, 1e-6)
    # the iterate is FP32 on output: error <= solve tolerance bound + FP32 rounding of V
    err = np.max(np.abs(v.double().cpu().numpy() - Vpi))
    assert err <= 1e-6 / (1 - mdp.gamma) + 2 ** -24 * np.max(np.abs(Vpi)) * 2
    # warm start from the exact solution: no Arnoldi step needed
    v2 = dev(Vpi)
    st2 = h.policy_eval(dev(pi), v2, 1e-8)
    assert st2["iters"] == 0 and st2["converged"]
    assert st["iters"] > 0
    h.close()


def test_policy_eval_banded_residual():
    mdp = synth.banded(40000, 4, 16, 2000, 0.5, 0.99, seed=22, dtype=np.float32)
    pi = np.random.default_rng(2).integers(0, mdp.m, size=mdp.n).astype(np.int32)
    h = _mk(mdp)
    v = torch.zeros(mdp.n, dtype=torch.float64, device="cuda")
    tol = 1e-8
    st = h.policy_eval(dev(pi), v, tol, restart=30)
    assert st["converged"]
    # the oracle's own FP64 evaluation of the residual has error ~ k eps |V| per entry
    slack = 64 * 2.0 ** -52 * 100 * np.sqrt(mdp.n)
    assert _policy_residual_2(mdp, pi, v.cpu().numpy()) <= tol * 1.01 + slack
    h.close()


def test_policy_eval_iteration_cap():
    mdp = synth.banded(20000, 4, 16, 2000, 0.5, 0.999, seed=23, dtype=np.float32)
    pi = np.zeros(mdp.n, dtype=np.int32)
    h = _mk(mdp)
    v = torch.zeros(mdp.n, dtype=torch.float64, device="cuda")
    st = h.policy_eval(dev(pi), v, 1e-14, restart=10, max_iters=25, raise_on_not_converged=False)
    assert st["status"] == "MDP_ERR_NOT_CONVERGED" and st["iters"] == 25
    assert np.isfinite(v.cpu().numpy()).all()
    h.close()


# ---------------------------------------------------------------------- solve

def test_solve_random_sparse_n1000_vs_exact_pi():
    mdp = synth.random_sparse_n1000()
    Vs, pis, _, _ = oracle.policy_iteration(mdp)
    h = _mk(mdp)
    tol = 1e-10
    V, pi, st = h.solve(tol=tol)
    Vg = V.cpu().numpy()
    assert st["converged"] and st["residual_inf"] <= tol
    assert np.max(np.abs(Vg - Vs)) <= tol / (1 - mdp.gamma) * 1.01
    cert = oracle.certificate(mdp, Vg)
    assert cert["res_inf"] <= tol * 1.01 + 1e-14
    clear = cert["gap"] > 2 * tol / (1 - mdp.gamma) + 1e-12
    assert np.array_equal(pi.cpu().numpy()[clear], pis[clear])
    h.close()


@pytest.mark.parametrize("inner", ["gmres", "richardson"])
def test_solve_inner_solvers_agree(inner):
    mdp = synth.random_sparse(2000, 4, 8, 1.0, 0.95, seed=31, dtype=np.float32)
    Vs, pis, _, _ = oracle.policy_iteration(mdp)
    h = _mk(mdp)
    tol = 1e-9
    V, pi, st = h.solve(tol=tol, inner=inner, max_inner=200)
    Vg = V.cpu().numpy()
    assert st["converged"]
    assert np.max(np.abs(Vg - Vs)) <= tol / (1 - mdp.gamma) * 1.01
    assert oracle.certificate(mdp, Vg)["res_inf"] <= tol * 1.01
    h.close()


def test_value_iteration_special_case():
    # iPI with a single Richardson sweep per outer step is value iteration:
    # its residuals contract by gamma per step (madupite: iPI contains VI)
    mdp = synth.random_sparse(500, 3, 6, 1.0, 0.8, seed=32, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9, inner="richardson", max_inner=1, max_outer=500)
    hist = np.array(st["residual_history"])
    assert st["converged"]
    assert np.all(hist[1:] <= mdp.gamma * hist[:-1] * (1 + 1e-5) + 1e-12)
    Vs, _, _, _ = oracle.policy_iteration(mdp)
    assert np.max(np.abs(V.cpu().numpy() - Vs)) <= 1e-9 / (1 - mdp.gamma) * 1.01
    h.close()


@pytest.mark.parametrize("store", ["f32", "bf16", "f16"])
def test_solve_grid_world_precision_path(store):
    """Low-precision inner solves refined by float-float outer residuals reach the
    FP32-P problem's 1e-9 residual; V matches exact PI on the same stored P."""
    mdp = synth.grid_world(33, 31, 0.999, seed=3, dtype=np.float32)
    Vs, _, _, _ = oracle.policy_iteration(mdp)
    h = _mk(mdp, store=store)
    tol = 1e-9
    V, pi, st = h.solve(tol=tol)
    Vg = V.cpu().numpy()
    assert st["converged"]
    cert = oracle.certificate(mdp, Vg)
    assert cert["res_inf"] <= tol * 1.05
    assert np.max(np.abs(Vg - Vs)) <= cert["res_inf"] / (1 - mdp.gamma) + 1e-9
    h.close()


def test_solve_warm_start_and_cgs2():
    mdp = synth.random_sparse(1500, 4, 8, 1.0, 0.99, seed=33, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9, cgs2=True)
    assert st["converged"]
    V2, pi2, st2 = h.solve(tol=1e-9, V_init=V)
    assert st2["outer_iters"] == 0 and torch.equal(V, V2) and torch.equal(pi, pi2)
    h.close()


def test_solve_banded_medium_certificate():
    mdp = synth.banded(65536, 8, 16, 4096, 0.5, 0.99, seed=2, dtype=np.float32)
    h = _mk(mdp)
    tol = 1e-9
    V, pi, st = h.solve(tol=tol)
    Vg = V.cpu().numpy()
    assert st["converged"] and st["outer_iters"] >= 1
    cert = oracle.certificate(mdp, Vg)
    assert cert["res_inf"] <= tol * 1.05
    clear = cert["gap"] > 2 * tol + 1e-12
    assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])
    h.close()


def test_solve_banded_small_vs_value_iteration():
    mdp = synth.banded(8192, 4, 16, 1024, 0.5, 0.99, seed=2, dtype=np.float32)
    h = _mk(mdp)
    V, pi, st = h.solve(tol=1e-9)
    Vg = V.cpu().numpy()
    Vv, piv, _, _ = oracle.value_iteration(mdp, 1e-9)
    assert st["converged"]
    # both within 1e-9 / (1 - gamma) of V*; VI's own bound is 1e-9
    assert np.max(np.abs(Vg - Vv)) <= 1e-9 / (1 - mdp.gamma) * 1.05 + 1e-9
    h.close()


def test_solve_banded_4m_full_size(banded_4m_gpu):
    """The full-size banded workload solved to a 1e-9 Bellman residual; the oracle
    certifies sampled blocks in FP64 (both band edges and the middle)."""
    mdp, h = banded_4m_gpu
    tol = 1e-9
    V, pi, st = h.solve(tol=tol)
    assert st["converged"] and st["residual_inf"] <= tol
    Vg = V.cpu().numpy()
    pig = pi.cpu().numpy()
    n = mdp.n
    for s0 in (0, n // 3, n - 4096):
        blk = synth.banded_4m(s0=s0, s1=s0 + 4096)
        cert = oracle.certificate(blk, Vg)
        assert cert["res_inf"] <= tol * 1.05
        clear = cert["gap"] > 2 * tol + 1e-12
        assert np.array_equal(pig[s0:s0 + 4096][clear], cert["pi"][clear])


@pytest.mark.parametrize("store", ["bf16", "f16"])
@pytest.mark.parametrize("packed", [True, False])
def test_solve_banded_low_precision_inner(store, packed, monkeypatch):
    """16-bit inner probabilities (packed 16-byte groups with int16 column offsets,
    or the plain 16-bit array) refined by the float-float outer residual reach
    the FP32-P problem's 1e-9 residual."""
    from paper_2502_14474_gb300 import MDP
    mdp = synth.banded(120000, 8, 16, 3000, 0.5, 0.99, seed=34, dtype=np.float32)
    if not packed:
        monkeypatch.setenv("MDP_NO_LP_PACK", "1")
    h = MDP.from_csr(mdp, store=store)
    monkeypatch.delenv("MDP_NO_LP_PACK", raising=False)
    assert h.info()["has_low_precision"]
    V, pi, st = h.solve(tol=1e-9)
    assert st["converged"]
    cert = oracle.certificate(mdp, V.cpu().numpy())
    assert cert["res_inf"] <= 1.05e-9
    clear = cert["gap"] > 2.1e-9
    assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])
    h.close()


def test_graph_replayed_cycles_match_eager():
    """Restart cycles replayed from captured CUDA graphs (side stream) give bitwise
    the same solve as eagerly launched cycles (legacy default stream)."""
    from paper_2502_14474_gb300 import MDP
    # large enough (2^20 states) for whole cycles, which smaller matrices enqueue
    # in chunks of eight steps instead
    mdp = synth.banded(1 << 20, 4, 16, 1500, 0.5, 0.99, seed=35, dtype=np.float32)
    eager = MDP.from_csr(mdp)
    Ve, pie, se = eager.solve(tol=1e-9)
    side = torch.cuda.Stream()
    g = MDP.from_csr(mdp, stream=side)
    Vg, pig, sg = g.solve(tol=1e-9)
    Vg2, pig2, sg2 = g.solve(tol=1e-9)  # second solve replays the cached graphs
    side.synchronize()
    assert torch.equal(Ve, Vg) and torch.equal(pie, pig)
    assert torch.equal(Vg, Vg2) and torch.equal(pig, pig2)
    assert se["inner_iters"] == sg["inner_iters"] == sg2["inner_iters"]
    eager.close()
    g.close()


@pytest.mark.parametrize("store", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["grid", "random"])
def test_action_major_policy_copy_is_bitwise_neutral(store, kind, monkeypatch):
    """Short rows are read by the policy-row kernels from an action-major copy
    padded with zero-probability entries; entries keep their order within a
    row, so every sum, hence every iterate, is bitwise what the CSR as given
    yields."""
    if kind == "grid":
        mdp = synth.grid_world(64, 48, 0.99, seed=5, dtype=np.float32)
    else:
        mdp = synth.random_sparse(3000, 4, 5, 1.0, 0.95, seed=6, k_max=6, dtype=np.float32)
    a = _mk(mdp, store=store)
    monkeypatch.setenv("MDP_NO_POLICY_COPY", "1")
    b = _mk(mdp, store=store)
    monkeypatch.delenv("MDP_NO_POLICY_COPY")
    # the copy exists only on the first handle
    assert a.info()["device_bytes"] > b.info()["device_bytes"]
    Va, pa, sa = a.solve(tol=1e-9)
    Vb, pb, sb = b.solve(tol=1e-9)
    assert sa["converged"] and sb["converged"]
    assert torch.equal(Va, Vb) and torch.equal(pa, pb)
    assert sa["inner_iters"] == sb["inner_iters"] and sa["outer_iters"] == sb["outer_iters"]
    cert = oracle.certificate(mdp, Va.cpu().numpy())
    assert cert["res_inf"] <= 1.05e-9
    a.close()
    b.close()


@pytest.mark.parametrize("s_step", [0, 6])
def test_profiler_counts_and_bytes_match_the_solve(s_step):
    """The event profiler behind the roofline numbers: one timed launch per
    executed policy SpMV and per sweep (classical Arnoldi: one dots and one
    orthogonalisation launch per step; s-step: one Gram and one update launch
    per block), the algorithmic bytes of the policy-row SpMV (4 action + 16 x 8
    packed row + 4 v_j + 4 w bytes per state), and percentiles that bracket the
    mean."""
    mdp = synth.banded(65536, 8, 16, 4096, 0.5, 0.99, seed=2, dtype=np.float32)
    h = _mk(mdp)
    h.profile(True)
    V, pi, st = h.solve(tol=1e-9, s_step=s_step)
    prof = h.profile_read()
    h.profile(False)
    k = prof["kinds"]
    assert st["converged"]
    assert k["arnoldi_spmv"]["launches"] == st["inner_iters"]
    if s_step == 0:
        assert k["arnoldi_dots"]["launches"] == st["inner_iters"]
        assert k["arnoldi_ortho"]["launches"] == st["inner_iters"]
        assert k["block_gram"]["launches"] == 0
    else:
        nb = k["block_gram"]["launches"]
        assert k["arnoldi_dots"]["launches"] == k["arnoldi_ortho"]["launches"] == 0
        assert k["block_update"]["launches"] == nb
        # every block but the last of a cycle ran all s SpMVs
        assert s_step * nb >= st["inner_iters"] > 0
        assert k["block_gram"]["bytes"] > 0 and k["block_update"]["bytes"] > 0
    assert k["bellman_ff"]["launches"] == st["bellman_sweeps"]
    assert k["policy_residual"]["launches"] == st["policy_sweeps"] - st["inner_iters"]
    sp = k["arnoldi_spmv"]
    assert sp["bytes"] == pytest.approx(sp["launches"] * 140.0 * mdp.n)
    mean = sp["ms"] / sp["launches"]
    assert 0 < sp["p50_ms"] <= sp["p99_ms"]
    assert sp["p50_ms"] <= 2 * mean and sp["p99_ms"] >= 0.5 * mean
    assert prof["total_launches"] >= sum(v["launches"] + v["skipped"] for v in k.values())
    h.close()


@pytest.mark.parametrize("store", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["random", "grid", "banded"])
def test_richardson_sweeps_stop_on_device(store, kind):
    """Modified PI enqueues Richardson sweeps eight at a time and each returns at
    once after one met the target: the sweeps that ran are exactly the policy
    sweeps counted, one inner step per outer iteration is the initial d = r.  The
    sweeps run through the policy-row kernel's Richardson form on every row layout
    (short rows with the action-major copy, banded rows with the ring window,
    packed 16-bit copies)."""
    if kind == "random":
        mdp = synth.random_sparse(3000, 4, 8, 1.0, 0.97, seed=34, dtype=np.float32)
    elif kind == "grid":
        mdp = synth.grid_world(48, 40, 0.97, seed=37, dtype=np.float32)
    else:
        mdp = synth.banded(40000, 4, 16, 1000, 0.5, 0.97, seed=38, dtype=np.float32)
    h = _mk(mdp, store=store)
    h.profile(True)
    V, pi, st = h.solve(tol=1e-9, inner="richardson", max_inner=500)
    k = h.profile_read()["kinds"]["richardson"]
    h.profile(False)
    assert st["converged"]
    assert k["launches"] == st["policy_sweeps"]
    assert st["inner_iters"] == st["policy_sweeps"] + st["outer_iters"]
    assert oracle.certificate(mdp, V.cpu().numpy())["res_inf"] <= 1.01e-9
    h.close()


def test_chunked_cycles_match_whole_cycles(monkeypatch):
    """Below 2^20 states a restart cycle is enqueued eight steps at a time with a
    status check between chunks; the steps that run, hence the solve, are
    bitwise those of a whole enqueued cycle."""
    from paper_2502_14474_gb300 import MDP
    mdp = synth.random_sparse(20000, 6, 8, 1.0, 0.99, seed=36, dtype=np.float32)
    a = MDP.from_csr(mdp)
    Va, pa, sa = a.solve(tol=1e-9)
    monkeypatch.setenv("MDP_NO_CYCLE_CHUNKS", "1")
    Vb, pb, sb = a.solve(tol=1e-9)
    monkeypatch.delenv("MDP_NO_CYCLE_CHUNKS")
    assert torch.equal(Va, Vb) and torch.equal(pa, pb)
    assert sa["inner_iters"] == sb["inner_iters"] and sa["outer_iters"] == sb["outer_iters"]
    a.close()

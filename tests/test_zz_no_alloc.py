"""The allocation-free Bellman entry point against the handle-based one.

mdp_bellman_noalloc serves callers that cannot allocate device memory: its
reduction scratch is a fixed file-scope device array, not a cudaMalloc.  It must
agree with mdp_bellman (FP32 path) on the same input, call after call (the
shared scratch is reused, so its ticket must be cleared every time).  This file
is collected last so that a failure here leaves every other test already run.
"""
import gc

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import check_greedy, dev, q_tol_f32

pytestmark = pytest.mark.gpu


def _inputs(mdp):
    return (dev(mdp.row_ptr), dev(mdp.col), dev(mdp.val.astype(np.float32)),
            dev(mdp.g.astype(np.float32)))


def test_noalloc_matches_handle_path_two_calls():
    from paper_2502_14474_gb300 import MDP, capi
    mdp = synth.banded(30011, 6, 12, 1500, 0.5, 0.99, seed=77, dtype=np.float32)
    rp, col, val, g = _inputs(mdp)
    h = MDP.from_csr(mdp)
    rng = np.random.default_rng(78)
    for call in range(2):
        V = rng.random(mdp.n).astype(np.float32) * (10.0 + 40.0 * call)
        Vt = dev(V)
        ref = h.bellman(Vt, want_r=True)
        V_out = torch.empty_like(Vt)
        pi_out = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
        r_out = torch.empty_like(Vt)
        res_inf, res_2 = capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, mdp.gamma, Vt,
                                                  V_out, pi_out, r_out,
                                                  stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        Vd = V.astype(np.float64)
        tol = q_tol_f32(mdp, Vd)
        # both paths are within tol of the exact T V, so within 2 tol of each other
        a = V_out.double().cpu().numpy()
        b = ref["V"].double().cpu().numpy()
        assert np.max(np.abs(a - b)) <= 2 * tol
        TV, pi, Q, _ = oracle.bellman(mdp, Vd, want_q=True)
        assert np.max(np.abs(a - TV)) <= tol  # the oracle's FP64 T V itself
        check_greedy(pi_out.cpu().numpy(), pi, Q, tol)
        ra = r_out.double().cpu().numpy()
        rb = ref["r"].double().cpu().numpy()
        rmax = float(np.max(np.abs(rb)))
        assert np.max(np.abs(ra - rb)) <= 2 * tol + 2.0 ** -23 * rmax
        assert abs(res_inf - ref["res_inf"]) <= 2 * tol + 2.0 ** -23 * rmax
        assert abs(res_2 - ref["res_2"]) <= (2 * tol + 2.0 ** -23 * rmax) * np.sqrt(mdp.n)
    h.close()


def test_noalloc_rejects_oversize_and_bad_columns():
    from paper_2502_14474_gb300 import capi
    from paper_2502_14474_gb300.capi import MDPError
    mdp = synth.random_sparse(1000, 2, 4, 1.0, 0.9, seed=79, dtype=np.float32)
    rp, col, val, g = _inputs(mdp)
    V = torch.zeros(mdp.n, device="cuda")
    with pytest.raises(MDPError) as ei:
        capi.mdp_bellman_noalloc(4194305, 1, rp, col, val, g, 0.9, V)
    assert ei.value.status_name == "MDP_ERR_ARG" and "4194304" in str(ei.value)
    bad = col.clone()
    bad[17] = mdp.n + 5
    with pytest.raises(MDPError) as ei:
        capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, bad, val, g, 0.9, V)
    assert ei.value.status_name == "MDP_ERR_BAD_CSR"
    # the shared scratch is usable again right after a failed call
    ri, _ = capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, 0.9, V)
    assert abs(ri - float(np.min(mdp.g.reshape(mdp.n, mdp.m), axis=1).max())) <= 1e-6


def test_noalloc_allocates_no_device_memory():
    """The property that defines the entry point: after a first call on the device
    (which may load the kernel's module), further calls change neither torch's
    allocator, nor the library's memory pool, nor the device's free memory."""
    from paper_2502_14474_gb300 import capi
    mdp = synth.random_sparse(20000, 4, 8, 1.0, 0.95, seed=80, dtype=np.float32)
    rp, col, val, g = _inputs(mdp)
    V = torch.rand(mdp.n, device="cuda")
    V_out = torch.empty_like(V)
    pi_out = torch.empty(mdp.n, dtype=torch.int32, device="cuda")
    r_out = torch.empty_like(V)
    s = torch.cuda.current_stream()
    capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, mdp.gamma, V, V_out, pi_out, r_out,
                             stream=s)
    torch.cuda.synchronize()
    gc.collect()  # tensors of earlier tests freed now, not during the calls below
    torch.cuda.synchronize()
    dev_i = torch.cuda.current_device()

    def snapshot():
        return (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
                capi.mdp_pool_trim(dev_i, 1 << 62), torch.cuda.mem_get_info()[0])
    before = snapshot()
    for _ in range(3):
        capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, mdp.gamma, V, V_out, pi_out,
                                 r_out, stream=s)
    torch.cuda.synchronize()
    after = snapshot()
    assert after[0] <= before[0]      # torch's allocator: nothing new
    assert after[1:] == before[1:]    # torch's reservation, the library pool, device memory


def test_noalloc_refuses_a_capturing_stream():
    """The call synchronises, so it refuses a stream that is capturing a graph
    (before it enqueues anything) instead of invalidating the caller's capture."""
    from paper_2502_14474_gb300 import capi
    from paper_2502_14474_gb300.capi import MDPError
    mdp = synth.random_sparse(1000, 2, 4, 1.0, 0.9, seed=81, dtype=np.float32)
    rp, col, val, g = _inputs(mdp)
    V = torch.zeros(mdp.n, device="cuda")
    capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, 0.9, V)  # device set-up first
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        V2 = V + 1.0
        torch.cuda.synchronize()
        with pytest.raises(MDPError) as ei:
            with torch.cuda.graph(graph, stream=s):
                V2.add_(1.0)
                capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, 0.9, V, stream=s)
    assert ei.value.status_name == "MDP_ERR_ARG"
    # the stream and the entry point are usable afterwards
    torch.cuda.synchronize()
    ri, _ = capi.mdp_bellman_noalloc(mdp.n, mdp.m, rp, col, val, g, 0.9, V)
    assert abs(ri - float(np.min(mdp.g.reshape(mdp.n, mdp.m), axis=1).max())) <= 1e-6

"""Batched solves, the autotuner and the serving loop on the GPU.

Every handle owns its device state and every reduction has a fixed order, so a
solve gives bitwise the same V and pi alone, in a concurrent batch, or among
the other requests of the serving loop.  The oracle certifies sampled results.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _uneven(count, seed, n_lo=2000, n_hi=20000):
    ps = synth.uneven_batch_params(count, seed=seed, n_lo=n_lo, n_hi=n_hi)
    return [synth.uneven_mdp(p) for p in ps]


def test_batch_solve_equals_individual_solves():
    from paper_2502_14474_gb300 import MDP, capi
    mdps = _uneven(10, seed=41)
    hs = [MDP.from_csr(m) for m in mdps]
    alone = [h.solve(tol=1e-9) for h in hs]
    Vs = [torch.empty(m.n, dtype=torch.float64, device="cuda") for m in mdps]
    pis = [torch.empty(m.n, dtype=torch.int32, device="cuda") for m in mdps]
    stats, status = capi.mdp_batch_solve([h.h for h in hs], Vs, pis, n_streams=4)
    assert all(s == "MDP_OK" for s in status)
    for (Va, pa, sa), Vb, pb, sb in zip(alone, Vs, pis, stats):
        assert torch.equal(Va, Vb) and torch.equal(pa, pb)
        assert sa["inner_iters"] == sb["inner_iters"] and sb["converged"]
    # oracle certificate on two of them
    for i in (0, 7):
        cert = oracle.certificate(mdps[i], Vs[i].cpu().numpy())
        assert cert["res_inf"] <= 1.05e-9
    for h in hs:
        h.close()


def test_autotune_keeps_the_answer():
    from paper_2502_14474_gb300 import MDP
    for mdp in (synth.banded(150000, 8, 16, 2000, 0.5, 0.99, seed=43, dtype=np.float32),
                _uneven(1, seed=44, n_lo=50000, n_hi=60000)[0]):
        a = MDP.from_csr(mdp)
        b = MDP.from_csr(mdp, autotune=True)
        Va, _, sa = a.solve(tol=1e-9)
        Vb, _, sb = b.solve(tol=1e-9)
        assert sa["converged"] and sb["converged"]
        assert b.info()["vec_width"] in (1, 2, 4, 8, 32)
        cert = oracle.certificate(mdp, Vb.cpu().numpy())
        assert cert["res_inf"] <= 1.05e-9
        assert np.max(np.abs(Va.cpu().numpy() - Vb.cpu().numpy())) <= 2.1e-9 / (1 - mdp.gamma)
        a.close()
        b.close()


def test_serving_results_identical_alone_and_in_the_mix():
    from paper_2502_14474_gb300 import MDP, serve
    mdps = _uneven(6, seed=45, n_lo=3000, n_hi=40000)
    arrivals = serve.poisson_arrivals(18, rate=400.0, seed=46)
    rng = np.random.default_rng(47)
    reqs = [serve.Request(rid=i, mdp=mdps[int(rng.integers(len(mdps)))], arrival=float(a))
            for i, a in enumerate(arrivals)]
    srv = serve.Server(budget_bytes=8e9, workers=4).start()
    wall = srv.run_trace(reqs)
    srv.close()
    summ = serve.summarize(reqs, wall)
    assert summ["completed"] == len(reqs), [r.error for r in reqs if r.status != "MDP_OK"]
    assert srv.peak_active >= 2 and srv.peak_used <= 8e9
    for k, mdp in enumerate(mdps):
        h = MDP.from_csr(mdp)
        V, pi, _ = h.solve(tol=1e-9)
        V, pi = V.cpu().numpy(), pi.cpu().numpy()
        h.close()
        for r in reqs:
            if r.mdp is mdp:
                assert np.array_equal(r.V, V) and np.array_equal(r.pi, pi)
    # the oracle's certificate of every distinct served MDP (a third of the requests)
    for mdp in mdps:
        r = next((q for q in reqs if q.mdp is mdp), None)
        if r is None:
            continue
        cert = oracle.certificate(mdp, r.V)
        assert cert["res_inf"] <= 1.05e-9
        assert cert["bound"] <= 1.05e-9 / (1 - mdp.gamma)


def test_serving_budget_admits_one_at_a_time():
    from paper_2502_14474_gb300 import serve
    mdps = _uneven(3, seed=48, n_lo=20000, n_hi=30000)
    srv = serve.Server(budget_bytes=1, workers=4)
    need = max(srv.request_bytes(serve.Request(rid=0, mdp=m)) for m in mdps)
    srv = serve.Server(budget_bytes=need * 1.5, workers=4).start()
    reqs = [serve.Request(rid=i, mdp=m) for i, m in enumerate(mdps * 2)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert all(r.status == "MDP_OK" for r in reqs)
    assert srv.peak_active == 1 and srv.peak_used <= need * 1.5


@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_bytes_required_bounds_the_handle(store):
    """Admission control reserves mdp_bytes_required per request: it must cover
    what a handle really holds (action-major copies of short rows included)."""
    from paper_2502_14474_gb300 import MDP, capi
    code = {"f32": capi.MDP_F32, "bf16": capi.MDP_BF16}[store]
    for mdp in (synth.banded(40000, 8, 16, 2000, 0.5, 0.99, seed=61, dtype=np.float32),
                synth.grid_world(96, 80, 0.99, seed=62, dtype=np.float32),
                synth.random_sparse(20000, 5, 4, 1.0, 0.95, seed=63, k_max=32, dtype=np.float32)):
        h = MDP.from_csr(mdp, store=store)
        held = h.info()["device_bytes"]
        need = capi.mdp_bytes_required(mdp.n, mdp.m, int(mdp.row_ptr[-1]), capi.MDP_F32, code, 30)
        assert need >= held, (mdp.name, need, held)
        h.close()

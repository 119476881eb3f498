"""Many MDPs with every solve phase in one launch (mdp_batch_solve_fused).

Each MDP's work units and reduction order depend only on that MDP, so its result
must be bitwise the same solved alone through the fused call and inside any
batch; the oracle certifies every result (FP64 ||T V - V||_inf within the
tolerance, greedy actions equal on clear Q-gaps).
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


def _fused(mdps, stream=None, autotune=False, **opts):
    from paper_2502_14474_gb300 import MDP, capi
    hs = [MDP.from_csr(m, autotune=autotune) for m in mdps]
    Vs = [torch.empty(m.n, dtype=torch.float64, device="cuda") for m in mdps]
    pis = [torch.empty(m.n, dtype=torch.int32, device="cuda") for m in mdps]
    o = capi.mdp_default_opts()
    o.tol = opts.get("tol", 1e-9)
    for k, v in opts.items():
        setattr(o, k, v)
    stats, status = capi.mdp_batch_solve_fused([h.h for h in hs], Vs, pis, opts=o, stream=stream)
    torch.cuda.synchronize()
    for h in hs:
        h.close()
    return Vs, pis, stats, status


def _certify(mdp, V, pi, tol=1e-9):
    cert = oracle.certificate(mdp, V.cpu().numpy())
    assert cert["res_inf"] <= tol * 1.05, cert["res_inf"]
    clear = cert["gap"] > 2 * tol + 1e-12
    assert np.array_equal(pi.cpu().numpy()[clear], cert["pi"][clear])


@pytest.mark.parametrize("graphs", [False, True])
def test_fused_batch_is_certified_and_equals_each_mdp_alone(graphs):
    mdps = _uneven(12, seed=61)
    stream = torch.cuda.Stream() if graphs else None
    Vs, pis, stats, status = _fused(mdps, stream=stream)
    assert all(s == "MDP_OK" for s in status), status
    for m, V, pi, st in zip(mdps, Vs, pis, stats):
        assert st["converged"] and st["residual_inf"] <= 1e-9
        _certify(m, V, pi)
    # alone through the fused call: bitwise the same V and pi, same work counts
    for i in (0, 5, 11):
        Va, pa, sa, _ = _fused([mdps[i]], stream=stream)
        assert torch.equal(Va[0], Vs[i]) and torch.equal(pa[0], pis[i])
        assert sa[0]["policy_sweeps"] == stats[i]["policy_sweeps"]
        assert sa[0]["outer_iters"] == stats[i]["outer_iters"]


def test_fused_batch_mixed_shapes_and_block_sizes():
    """Banded rows (uniform length), grid rows (short, uneven), random rows, an
    autotuned lane count, and the block sizes 1, 4 and 8."""
    mdps = [synth.banded(30000, 8, 16, 2000, 0.5, 0.99, seed=62, dtype=np.float32),
            synth.grid_world(101, 97, 0.99, 63, dtype=np.float32),
            synth.random_sparse(7001, 3, 9, 1.0, 0.97, seed=64, dtype=np.float32)]
    for s_step in (1, 4, 8):
        Vs, pis, stats, status = _fused(mdps, stream=torch.cuda.Stream(), autotune=True,
                                        s_step=s_step)
        assert all(s == "MDP_OK" for s in status), (s_step, status)
        for m, V, pi in zip(mdps, Vs, pis):
            _certify(m, V, pi)


def test_fused_batch_matches_the_single_solve_within_tolerance():
    from paper_2502_14474_gb300 import MDP
    mdps = _uneven(4, seed=65)
    Vs, pis, stats, status = _fused(mdps)
    for m, V in zip(mdps, Vs):
        h = MDP.from_csr(m)
        V1, _, _ = h.solve(tol=1e-9)
        h.close()
        # both within 1e-9 / (1 - gamma) of V*
        bound = 1.05e-9 / (1 - m.gamma)
        assert torch.max(torch.abs(V - V1)).item() <= 2 * bound


def test_fused_batch_rejects_what_it_does_not_run():
    from paper_2502_14474_gb300 import MDP, MDPError, capi
    m = _uneven(1, seed=66)[0]
    h = MDP.from_csr(m)
    V = torch.empty(m.n, dtype=torch.float64, device="cuda")
    o = capi.mdp_default_opts()
    o.cgs2, o.s_step = 1, 0
    with pytest.raises(MDPError):
        capi.mdp_batch_solve_fused([h.h], [V], opts=o)
    with pytest.raises(MDPError):
        capi.mdp_batch_solve_fused([h.h, h.h], [V, V])
    o = capi.mdp_default_opts()
    o.inner = capi.MDP_INNER_RICHARDSON
    with pytest.raises(MDPError):
        capi.mdp_batch_solve_fused([h.h], [V], opts=o)
    h.close()

"""GPU tests of cancellation: mdp_cancel from another thread stops a running
solve at its next host check (MDP_ERR_CANCELLED) and leaves the handle usable;
the serving loop cancels a running request through it and drops a queued one.
The solves are made long on purpose: an inner target of 1e-30 times the
residual keeps GMRES running to max_inner (a million Arnoldi steps, seconds)
inside the first outer iteration, whatever the outer residual does; the
cancel lands there.  max_outer = 2 bounds the solve, so a cancel that failed
to land ends in MDP_ERR_NOT_CONVERGED instead of a hang."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

LONG = dict(tol=0.0, inner_rtol=1e-30, max_outer=2, max_inner=1_000_000)

pytestmark = pytest.mark.gpu


def _wait(cond, seconds):
    t0 = time.perf_counter()
    while not cond() and time.perf_counter() - t0 < seconds:
        time.sleep(0.005)
    return cond()


def test_mdp_cancel_stops_a_running_solve():
    from paper_2502_14474_gb300 import MDP, MDPError, capi
    mdp = synth.random_sparse(20000, 4, 8, 1.0, 0.99, seed=71, dtype=np.float32)
    h = MDP.from_csr(mdp)
    out = {}

    def run():
        try:
            h.solve(**LONG)
            out["status"] = "finished"
        except MDPError as e:
            out["status"] = e.status_name

    t = threading.Thread(target=run)
    t.start()
    time.sleep(0.3)
    assert "status" not in out          # still running
    capi.mdp_cancel(h.h)
    t.join(timeout=60)
    assert not t.is_alive() and out["status"] == "MDP_ERR_CANCELLED"
    # the handle is not broken: the next solve runs to the tolerance
    V, pi, st = h.solve(tol=1e-9)
    assert st["converged"]
    assert oracle.certificate(mdp, V.cpu().numpy())["res_inf"] <= 1.01e-9
    h.close()


def test_serving_cancels_running_and_queued_requests():
    from paper_2502_14474_gb300 import serve
    mdp = synth.random_sparse(20000, 4, 8, 1.0, 0.99, seed=72, dtype=np.float32)
    srv = serve.Server(budget_bytes=50e9, workers=1,
                       solve_opts=LONG).start()
    a, b = serve.Request(rid=0, mdp=mdp), serve.Request(rid=1, mdp=mdp)
    srv.submit(a)
    srv.submit(b)
    assert _wait(lambda: a.handle is not None, 60)   # a is solving, b waits
    assert srv.cancel(b) and b.status == "MDP_ERR_CANCELLED"
    time.sleep(0.2)
    assert srv.cancel(a)
    assert _wait(lambda: a.t_done > 0, 120)
    srv.close()
    assert a.status == "MDP_ERR_CANCELLED", a.error
    assert srv.used == 0 and srv.active == 0


def test_cancel_before_the_call_is_honoured_once():
    """A cancel request made while no call runs stays pending: the next solve (or
    policy evaluation) returns MDP_ERR_CANCELLED at once, which consumes it, and
    the call after that runs normally."""
    import torch
    from paper_2502_14474_gb300 import MDP, MDPError, capi
    mdp = synth.random_sparse(5000, 4, 8, 1.0, 0.95, seed=73, dtype=np.float32)
    h = MDP.from_csr(mdp)
    capi.mdp_cancel(h.h)
    with pytest.raises(MDPError) as ei:
        h.solve(tol=1e-9)
    assert ei.value.status_name == "MDP_ERR_CANCELLED"
    V, pi, st = h.solve(tol=1e-9)
    assert st["converged"]
    assert oracle.certificate(mdp, V.cpu().numpy())["res_inf"] <= 1.01e-9
    capi.mdp_cancel(h.h)
    v = torch.zeros(mdp.n, dtype=torch.float64, device="cuda")
    with pytest.raises(MDPError) as ei:
        h.policy_eval(pi, v, tol=1e-8)
    assert ei.value.status_name == "MDP_ERR_CANCELLED"
    st2 = h.policy_eval(pi, v, tol=1e-8)
    assert st2["converged"]
    h.close()

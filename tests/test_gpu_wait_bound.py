"""Bounded barrier waits of the bulk-copy Gram pass.

Every mbarrier wait of `k_block_gram` gives up after 2 s of global time, marks
the launch in the device state, and the next status read turns that into
MDP_ERR_TIMEOUT.  The test switch MDP_TEST_STALL_GRAM keeps the producer from
arming any stage -- a barrier that nothing completes, with no copy in flight --
so the consumers' waits run out.  The solve must fail with MDP_ERR_TIMEOUT
within seconds, and the context and the handle must stay usable: the same handle
then solves correctly (the oracle certifies it).
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_gram_wait_timeout_is_reported_and_the_handle_recovers(monkeypatch):
    from paper_2502_14474_gb300 import MDP, MDPError
    mdp = synth.banded(40000, 8, 16, 800, 0.5, 0.99, seed=401, dtype=np.float32)
    h = MDP.from_csr(mdp)
    monkeypatch.setenv("MDP_TEST_STALL_GRAM", "1")
    t0 = time.time()
    with pytest.raises(MDPError) as ei:
        h.solve(tol=1e-9, s_step=6)
    took = time.time() - t0
    monkeypatch.delenv("MDP_TEST_STALL_GRAM")
    assert ei.value.status_name == "MDP_ERR_TIMEOUT", str(ei.value)
    assert 1.5 <= took <= 60.0, took
    V, pi, st = h.solve(tol=1e-9, s_step=6)
    assert st["converged"]
    cert = oracle.certificate(mdp, V.cpu().numpy())
    assert cert["res_inf"] <= 1.05e-9
    h.close()

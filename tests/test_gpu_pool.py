"""The library's device memory pool: destroyed handles leave their memory
cached for reuse, mdp_pool_trim hands it back, live handles keep theirs."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_pool_reuse_and_trim():
    from paper_2502_14474_gb300 import MDP, capi
    mdp = synth.banded(200000, 4, 8, 1000, 0.5, 0.95, seed=91, dtype=np.float32)
    a = MDP.from_csr(mdp)
    Va, pa, _ = a.solve(tol=1e-9)
    held = a.info()["device_bytes"]
    # a live handle's memory is never released (other live handles of this
    # process may hold more of the pool)
    r_live = capi.mdp_pool_trim(0, 0)
    assert r_live >= held
    a.close()
    # cached after destroy, released by the trim (pool chunks that the handle
    # shared with live allocations of other handles stay reserved)
    assert capi.mdp_pool_trim(0, 1 << 62) >= r_live
    assert capi.mdp_pool_trim(0, 0) <= r_live - 0.5 * held
    # a handle created after the trim gets fresh memory and the same answer
    b = MDP.from_csr(mdp)
    Vb, pb, _ = b.solve(tol=1e-9)
    assert np.array_equal(Va.cpu().numpy(), Vb.cpu().numpy())
    assert np.array_equal(pa.cpu().numpy(), pb.cpu().numpy())
    b.close()


def test_pool_trim_rejects_bad_device():
    from paper_2502_14474_gb300 import capi
    from paper_2502_14474_gb300.capi import MDPError
    with pytest.raises(MDPError) as ei:
        capi.mdp_pool_trim(-1, 0)
    assert ei.value.status_name == "MDP_ERR_ARG"

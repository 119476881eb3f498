"""Seeded workload generators: known-answer RNG, structure of each workload."""
import numpy as np

import synth


def test_philox_known_answers():
    # Philox4x32-10 known-answer vectors (Salmon et al., SC 2011; Random123 kat_vectors)
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C,
                                                          0x9B00DBD8]
    assert synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E,
                                                                     0xA20BC7C6, 0x6D5451FD]
    assert synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                               [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420,
                                                             0x24126EA1]


def _check_csr(mdp, tol):
    rp, col = mdp.row_ptr, mdp.col
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1)
    assert col.min() >= 0 and col.max() < mdp.n
    for r in range(min(mdp.rows, 2000)):
        c = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.all(mdp.val > 0)
    sums = np.add.reduceat(mdp.val.astype(np.float64), rp[:-1])
    assert np.max(np.abs(sums - 1)) <= tol


def test_random_sparse_structure():
    mdp = synth.random_sparse_n1000()
    assert mdp.nnz == 1000 * 4 * 8
    _check_csr(mdp, 1e-12)
    assert 0 <= mdp.g.min() and mdp.g.max() <= 1


def test_banded_structure_and_determinism():
    a = synth.banded(20000, 8, 16, 4096, 0.5, 0.99, seed=2, dtype=np.float32)
    _check_csr(a, 1e-5)
    s = np.repeat(np.arange(a.n), a.m * 16)
    assert np.all(np.abs(a.col.astype(np.int64) - s) <= 4096)
    b = synth.banded(20000, 8, 16, 4096, 0.5, 0.99, seed=2, dtype=np.float32, s0=5000, s1=6000)
    e0, e1 = a.row_ptr[5000 * 8], a.row_ptr[6000 * 8]
    assert np.array_equal(b.col, a.col[e0:e1]) and np.array_equal(b.val, a.val[e0:e1])
    assert np.array_equal(b.g, a.g[5000 * 8:6000 * 8])


def test_uneven_row_lengths():
    p = dict(n=3000, m=5, k_min=4, k_max=32, alpha=1.0, gamma=0.95, seed=99)
    mdp = synth.uneven_mdp(p)
    lens = np.diff(mdp.row_ptr)
    assert lens.min() >= 4 and lens.max() <= 32 and len(np.unique(lens)) > 20
    _check_csr(mdp, 1e-5)


def test_grid_world_structure():
    W = 16
    mdp = synth.grid_world(W, W, 0.999, seed=3, dtype=np.float64)
    _check_csr(mdp, 1e-12)
    lens = np.diff(mdp.row_ptr).reshape(W * W, 5)
    assert lens.max() == 5 and lens[0].max() == 3  # corner rows merge two walls
    goals = synth.grid_goals(W, W, 16, 3)
    assert len(set(goals.tolist())) == 16
    g = mdp.g.reshape(-1, 5)
    assert np.all(g[goals] == 0) and g.sum() == 5 * (W * W - 16)
    # intended move east from an interior cell
    s = 5 * W + 5
    r = s * 5 + 1
    c = mdp.col[mdp.row_ptr[r]:mdp.row_ptr[r + 1]]
    v = mdp.val[mdp.row_ptr[r]:mdp.row_ptr[r + 1]]
    assert list(c) == [s - W, s - 1, s, s + 1, s + W]
    assert np.allclose(v, [0.05, 0.05, 0.05, 0.8, 0.05])


def test_uneven_batch_params():
    ps = synth.uneven_batch_params(512)
    ns = np.array([p["n"] for p in ps])
    assert ns.min() >= 2000 and ns.max() <= 200000
    assert {p["m"] for p in ps} <= set(range(2, 17))
    assert all(0.9 <= p["gamma"] <= 0.999 for p in ps)

"""Host-side MDP ingest (include/mdp_ingest.h): runs on the CPU, no GPU.

Each builder is checked against an independent construction:
* from_functions: the CSR built by hand from the same generator (sorted rows,
  repeated successors summed), for several thread counts;
* from_samples: the maximum-likelihood model counted in plain Python
  (P = N(s,a,s')/N(s,a), g = mean cost in sample order), exactly;
* read_petsc: files encoded here with struct from the PETSc binary matrix
  layout (big-endian header {1211216, rows, cols, nz or -1}, row lengths,
  column indices, values), in 32- and 64-bit integer widths, dense and sparse
  costs, unsorted rows with repeated columns; and write/read round trips.
"""
import collections
import os
import struct

import numpy as np
import pytest

import synth

CLASS_ID = 1211216


@pytest.fixture(scope="module")
def ingest():
    from paper_2502_14474_gb300 import ingest as mod
    return mod


def _gen(n, m, seed):
    """A deterministic generator with unsorted, repeated successors."""
    def transitions(s, a):
        rng = np.random.default_rng(seed * 1_000_003 + s * 31 + a)
        k = 1 + (s + a) % 7
        succ = rng.integers(0, n, size=k)
        w = rng.random(k) + 0.1
        return succ.tolist(), (w / w.sum()).tolist()

    def cost(s, a):
        return float(np.sin(s + 0.25 * a))
    return transitions, cost


def _by_hand(n, m, transitions, cost):
    row_ptr, col, val, g = [0], [], [], []
    for s in range(n):
        for a in range(m):
            succ, prob = transitions(s, a)
            acc = collections.OrderedDict()
            for c, p in sorted(zip(succ, prob), key=lambda t: t[0]):  # stable: equal keys in order
                acc[c] = acc.get(c, 0.0) + p
            col += list(acc.keys())
            val += list(acc.values())
            row_ptr.append(len(col))
            g.append(cost(s, a))
    return (np.array(row_ptr, np.int64), np.array(col, np.int32), np.array(val, np.float64),
            np.array(g, np.float64))


def _same(h, ref):
    for x, y in zip((h.row_ptr, h.col, h.val, h.g), ref):
        assert x.dtype == y.dtype and np.array_equal(x, y)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_from_functions_matches_hand_built_csr(ingest, threads):
    n, m = 40, 3
    tr, cost = _gen(n, m, seed=1)
    h = ingest.from_functions(n, m, tr, cost, gamma=0.9, threads=threads)
    assert (h.n, h.m, h.gamma) == (n, m, 0.9)
    _same(h, _by_hand(n, m, tr, cost))


def test_from_functions_long_rows_are_requested_again(ingest):
    n, m = 300, 2  # rows of 200 entries exceed the library's first buffer

    def tr(s, a):
        succ = [(s + 7 * i) % n for i in range(200)]
        return succ, [1.0 / 200] * 200
    h = ingest.from_functions(n, m, tr, lambda s, a: 1.0, gamma=0.5)
    _same(h, _by_hand(n, m, tr, lambda s, a: 1.0))


def test_from_functions_errors(ingest):
    from paper_2502_14474_gb300 import MDPError
    ok = lambda s, a: ([s], [1.0])  # noqa: E731
    with pytest.raises(MDPError, match="BAD_CSR.*successor 9 of .s, a. = .2, 1."):
        ingest.from_functions(5, 2, lambda s, a: ([9], [1.0]) if (s, a) == (2, 1) else ok(s, a),
                              lambda s, a: 0.0, 0.9)
    with pytest.raises(MDPError, match="NOT_STOCHASTIC.*negative"):
        ingest.from_functions(5, 2, lambda s, a: ([s], [-1.0]), lambda s, a: 0.0, 0.9)
    with pytest.raises(MDPError, match="NOT_STOCHASTIC.*no successor"):
        ingest.from_functions(5, 2, lambda s, a: ([], []), lambda s, a: 0.0, 0.9)
    with pytest.raises(MDPError, match="NONFINITE.*cost"):
        ingest.from_functions(5, 2, ok, lambda s, a: float("inf"), 0.9)
    with pytest.raises(MDPError, match="NONFINITE.*probability"):
        ingest.from_functions(5, 2, lambda s, a: ([s], [float("nan")]), lambda s, a: 0.0, 0.9)
    with pytest.raises(ZeroDivisionError):
        ingest.from_functions(5, 2, lambda s, a: 1 / 0, lambda s, a: 0.0, 0.9)
    with pytest.raises(KeyError):
        ingest.from_functions(5, 2, ok, lambda s, a: {}[s], 0.9)
    with pytest.raises(ValueError, match="successors"):
        ingest.from_functions(5, 2, lambda s, a: ([1, 2], [1.0]), lambda s, a: 0.0, 0.9)
    with pytest.raises(MDPError, match="ARG"):
        ingest.from_functions(0, 2, ok, lambda s, a: 0.0, 0.9)


@pytest.mark.parametrize("threads", [1, 4, 16])
def test_from_functions_reports_the_lowest_failing_row(ingest, threads):
    from paper_2502_14474_gb300 import MDPError

    def tr(s, a):
        return ([-5], [1.0]) if s in (11, 57, 90) else ([s], [1.0])
    with pytest.raises(MDPError, match=r"successor -5 of \(s, a\) = \(11, 0\)"):
        ingest.from_functions(100, 2, tr, lambda s, a: 0.0, 0.9, threads=threads)


def _ml_by_hand(n, m, s, a, sn, c, unseen_cost=None):
    cnt = collections.defaultdict(collections.Counter)
    csum = collections.defaultdict(list)
    for i in range(len(s)):
        cnt[(s[i], a[i])][sn[i]] += 1
        csum[(s[i], a[i])].append(c[i])
    row_ptr, col, val, g = [0], [], [], []
    for st in range(n):
        for ac in range(m):
            N = sum(cnt[(st, ac)].values())
            if N == 0:
                col.append(st)
                val.append(1.0)
                g.append(unseen_cost)
            else:
                for nx in sorted(cnt[(st, ac)]):
                    col.append(nx)
                    val.append(cnt[(st, ac)][nx] / N)
                acc = 0.0
                for x in csum[(st, ac)]:  # plain left-to-right sum (builtin sum() compensates)
                    acc += x
                g.append(acc / N)
            row_ptr.append(len(col))
    return (np.array(row_ptr, np.int64), np.array(col, np.int32), np.array(val, np.float64),
            np.array(g, np.float64))


@pytest.mark.parametrize("threads", [1, 5])
def test_from_samples_is_the_counting_estimator(ingest, threads):
    rng = np.random.default_rng(7)
    n, m, count = 30, 4, 5000
    s = rng.integers(0, n, count)
    a = rng.integers(0, m, count)
    sn = (s + rng.integers(-3, 4, count)) % n
    c = rng.normal(size=count)
    h = ingest.from_samples(n, m, s, a, sn, c, gamma=0.8, threads=threads)
    _same(h, _ml_by_hand(n, m, s.tolist(), a.tolist(), sn.tolist(), c.tolist()))
    assert np.allclose(np.add.reduceat(h.val, h.row_ptr[:-1]), 1.0, atol=1e-14)


def test_from_samples_unseen_pairs(ingest):
    from paper_2502_14474_gb300 import MDPError
    s, a, sn, c = [0, 0, 2], [1, 1, 0], [1, 2, 2], [1.0, 3.0, 5.0]
    with pytest.raises(MDPError, match=r"no sample of \(s, a\) = \(0, 0\)"):
        ingest.from_samples(3, 2, s, a, sn, c)
    h = ingest.from_samples(3, 2, s, a, sn, c, unseen="self_loop", unseen_cost=9.0)
    _same(h, _ml_by_hand(3, 2, s, a, sn, c, unseen_cost=9.0))
    assert h.g.tolist() == [9.0, 2.0, 9.0, 9.0, 5.0, 9.0]
    with pytest.raises(MDPError, match="sample 1"):
        ingest.from_samples(3, 2, [0, 3], [0, 0], [0, 0], [0.0, 0.0], unseen="self_loop")
    with pytest.raises(MDPError, match="NONFINITE.*sample 0"):
        ingest.from_samples(3, 2, [0], [0], [0], [float("nan")], unseen="self_loop")
    h0 = ingest.from_samples(2, 1, [0, 1], [0, 0], [1, 0], None)
    assert h0.g.tolist() == [0.0, 0.0]


# ------------------------------------------------------------- PETSc files

def _aij(rows, cols, rowlens, colidx, vals, w=4):
    it = ">i" if w == 4 else ">q"
    out = b"".join(struct.pack(it, x) for x in (CLASS_ID, rows, cols, len(colidx)))
    out += b"".join(struct.pack(it, x) for x in rowlens)
    out += b"".join(struct.pack(it, x) for x in colidx)
    out += b"".join(struct.pack(">d", x) for x in vals)
    return out


def _dense(rows, cols, vals, w=4):
    it = ">i" if w == 4 else ">q"
    out = b"".join(struct.pack(it, x) for x in (CLASS_ID, rows, cols, -1))
    return out + b"".join(struct.pack(">d", x) for x in vals)


def _write(tmp_path, name, data):
    p = os.path.join(tmp_path, name)
    with open(p, "wb") as fh:
        fh.write(data)
    return p


@pytest.mark.parametrize("w", [4, 8])
def test_read_petsc_hand_encoded(ingest, tmp_path, w):
    # n = 3 states, m = 2 actions; row 1 unsorted with a repeated column
    rowlens = [1, 3, 2, 1, 1, 2]
    colidx = [0, 2, 0, 2, 1, 2, 1, 0, 1, 0]
    vals = [1.0, 0.25, 0.5, 0.25, 0.5, 0.5, 1.0, 1.0, 0.75, 0.25]
    p = _write(tmp_path, "P.bin", _aij(6, 3, rowlens, colidx, vals, w))
    g = _write(tmp_path, "g.bin", _dense(3, 2, [1.0, 2.0, 3.0, 4.0, 5.0, 6.0], w))
    h = ingest.read_petsc(p, g, gamma=0.7)
    assert (h.n, h.m, h.nnz) == (3, 2, 9)
    assert h.row_ptr.tolist() == [0, 1, 3, 5, 6, 7, 9]
    assert h.col.tolist() == [0, 0, 2, 1, 2, 1, 0, 0, 1]
    assert h.val.tolist() == [1.0, 0.5, 0.5, 0.5, 0.5, 1.0, 1.0, 0.25, 0.75]
    assert h.g.tolist() == [1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
    # sparse costs: missing entries are 0, repeated ones summed
    gs = _write(tmp_path, "gs.bin", _aij(3, 2, [2, 0, 1], [1, 1, 0], [2.0, 0.5, -1.0], w))
    hs = ingest.read_petsc(p, gs)
    assert hs.g.tolist() == [0.0, 2.5, 0.0, 0.0, -1.0, 0.0]
    assert ingest.read_petsc(p).g.tolist() == [0.0] * 6


def test_read_petsc_rejects_bad_files(ingest, tmp_path):
    from paper_2502_14474_gb300 import MDPError
    good = _aij(2, 1, [1, 1], [0, 0], [1.0, 1.0])
    p = _write(tmp_path, "P.bin", good)
    with pytest.raises(MDPError, match="truncated"):
        ingest.read_petsc(_write(tmp_path, "T.bin", good[:-3]))
    with pytest.raises(MDPError, match="not a PETSc binary matrix"):
        ingest.read_petsc(_write(tmp_path, "X.bin", b"\x00\x00\x00\x07" + good[4:]))
    with pytest.raises(MDPError, match="n\\*m rows"):
        ingest.read_petsc(_write(tmp_path, "R.bin", _aij(3, 2, [1, 1, 1], [0, 0, 0], [1.0] * 3)))
    with pytest.raises(MDPError, match="BAD_CSR"):
        ingest.read_petsc(_write(tmp_path, "C.bin", _aij(2, 1, [1, 1], [0, 1], [1.0, 1.0])))
    with pytest.raises(MDPError, match="do not add up"):
        ingest.read_petsc(_write(tmp_path, "L.bin", _aij(2, 1, [1, 2], [0, 0], [1.0, 1.0])))
    with pytest.raises(MDPError, match="NONFINITE"):
        ingest.read_petsc(_write(tmp_path, "N.bin", _aij(2, 1, [1, 1], [0, 0],
                                                          [1.0, float("inf")])))
    with pytest.raises(MDPError, match="costs are 2 x 2"):
        ingest.read_petsc(p, _write(tmp_path, "g.bin", _dense(2, 2, [0.0] * 4)))
    with pytest.raises(MDPError, match="cannot open"):
        ingest.read_petsc(os.path.join(tmp_path, "missing.bin"))
    with pytest.raises(MDPError, match="sparse"):
        ingest.read_petsc(_write(tmp_path, "D.bin", _dense(2, 1, [1.0, 1.0])))


def test_write_read_round_trip(ingest, tmp_path):
    mdp = synth.banded(500, 4, 6, 20, 0.5, 0.95, seed=3, dtype=np.float32)
    p, g = os.path.join(tmp_path, "P.bin"), os.path.join(tmp_path, "g.bin")
    ingest.write_petsc(mdp, p, g)
    nnz, rows = mdp.nnz, mdp.n * mdp.m
    assert os.path.getsize(p) == 16 + 4 * rows + 12 * nnz
    assert os.path.getsize(g) == 16 + 8 * rows
    h = ingest.read_petsc(p, g, gamma=mdp.gamma, threads=3)
    assert (h.n, h.m) == (mdp.n, mdp.m)
    assert np.array_equal(h.row_ptr, mdp.row_ptr) and np.array_equal(h.col, mdp.col)
    assert np.array_equal(h.val, mdp.val.astype(np.float64))
    assert np.array_equal(h.g, mdp.g.astype(np.float64))
    # a HostMDP writes back to the same bytes
    p2 = os.path.join(tmp_path, "P2.bin")
    ingest.write_petsc(h, p2)
    assert open(p, "rb").read() == open(p2, "rb").read()
    # the 32-bit file agrees with a hand encoding of the first rows' layout
    raw = open(p, "rb").read()
    assert struct.unpack(">4i", raw[:16]) == (CLASS_ID, rows, mdp.n, nnz)
    lens = np.frombuffer(raw[16:16 + 4 * rows], dtype=">i4")
    assert np.array_equal(lens, np.diff(mdp.row_ptr))


def test_read_petsc_survives_corrupt_files(ingest, tmp_path):
    """Seeded fuzzing: truncations and byte flips of valid files (header, row
    lengths, columns, values; 32- and 64-bit; sparse and dense costs).  Each read
    either raises MDPError or returns a structurally valid CSR -- it never
    crashes or reads past the file."""
    from paper_2502_14474_gb300 import MDPError
    rng = np.random.default_rng(2024)
    rowlens = [1, 3, 2, 1, 1, 2]
    colidx = [0, 2, 0, 2, 1, 2, 1, 0, 1, 0]
    vals = [1.0, 0.25, 0.5, 0.25, 0.5, 0.5, 1.0, 1.0, 0.75, 0.25]
    bases = [(_aij(6, 3, rowlens, colidx, vals, w), g)
             for w in (4, 8)
             for g in (_dense(3, 2, [1.0, 2.0, 3.0, 4.0, 5.0, 6.0], w),
                       _aij(3, 2, [2, 0, 1], [1, 1, 0], [2.0, 0.5, -1.0], w))]
    ok = failed = 0
    for trial in range(400):
        P, G = bases[trial % len(bases)]
        P, G = bytearray(P), bytearray(G)
        target = P if rng.random() < 0.7 else G
        kind = rng.integers(3)
        if kind == 0:      # truncate
            del target[int(rng.integers(0, len(target))):]
        elif kind == 1:    # flip bytes
            for _ in range(int(rng.integers(1, 4))):
                target[int(rng.integers(0, len(target)))] ^= int(rng.integers(1, 256))
        else:              # overwrite a header integer with an extreme value
            w = 4 if P[:4] == struct.pack(">i", CLASS_ID) else 8
            slot = int(rng.integers(1, 4))
            v = int(rng.choice([-2, -1, 0, 2**31 - 1, 2**30, 7]))
            fmt = ">i" if w == 4 else ">q"
            target[slot * w:(slot + 1) * w] = struct.pack(fmt, v)
        p = _write(tmp_path, "fP.bin", bytes(P))
        g = _write(tmp_path, "fg.bin", bytes(G))
        try:
            h = ingest.read_petsc(p, g)
        except MDPError:
            failed += 1
            continue
        ok += 1
        assert h.row_ptr[0] == 0 and np.all(np.diff(h.row_ptr) >= 0)
        assert h.row_ptr[-1] == h.nnz == h.col.size == h.val.size
        assert np.all((h.col >= 0) & (h.col < h.n))
        assert np.all(np.isfinite(h.val)) and np.all(np.isfinite(h.g))
        for r in range(h.rows):
            c = h.col[h.row_ptr[r]:h.row_ptr[r + 1]]
            assert np.all(np.diff(c) > 0)
    assert failed > 100 and ok > 20


def test_npz_round_trip(ingest, tmp_path):
    mdp = synth.random_sparse(300, 3, 5, 1.0, 0.9, seed=8, dtype=np.float32)
    p = os.path.join(tmp_path, "mdp.npz")
    ingest.save_npz(mdp, p)
    h = ingest.load_npz(p)
    assert (h.n, h.m, h.gamma, h.maximize) == (mdp.n, mdp.m, mdp.gamma, False)
    for a, b in ((h.row_ptr, mdp.row_ptr), (h.col, mdp.col), (h.val, mdp.val), (h.g, mdp.g)):
        assert a.dtype == b.dtype and np.array_equal(a, b)
    h2 = ingest.HostMDP(n=h.n, m=h.m, gamma=0.5, row_ptr=h.row_ptr, col=h.col,
                        val=h.val.astype(np.float64), g=-h.g.astype(np.float64), maximize=True)
    ingest.save_npz(h2, p)
    h3 = ingest.load_npz(p)
    assert h3.maximize and h3.gamma == 0.5 and h3.val.dtype == np.float64
    np.savez(p, n=3, m=1, gamma=0.9, row_ptr=np.arange(3), col=np.zeros(2), val=np.ones(2),
             g=np.zeros(3))
    with pytest.raises(ValueError, match="n\\*m\\+1"):
        ingest.load_npz(p)


# module-level generators: picklable for the worker processes of from_functions
def _sim_transitions(s, a):
    rng = np.random.default_rng(7_000_003 + s * 31 + a)
    k = 1 + (s + 2 * a) % 6
    succ = rng.integers(0, 60, size=k)
    w = rng.random(k) + 0.05
    return succ.tolist(), (w / w.sum()).tolist()


def _sim_cost(s, a):
    return float(np.cos(0.3 * s + a))


def _sim_fails(s, a):
    if s == 37:
        raise RuntimeError("simulator failed at state 37")
    return [s], [1.0]


def _raw_rows(n, m, transitions, cost):
    offsets, col, prob, g = [0], [], [], []
    for s in range(n):
        for a in range(m):
            succ, p = transitions(s, a)
            col += list(succ)
            prob += list(p)
            offsets.append(len(col))
            g.append(cost(s, a))
    return np.array(offsets), np.array(col), np.array(prob), np.array(g)


@pytest.mark.parametrize("threads", [1, 4])
def test_from_rows_equals_from_functions(ingest, threads):
    n, m = 60, 3
    ref = ingest.from_functions(n, m, _sim_transitions, _sim_cost, gamma=0.9)
    h = ingest.from_rows(n, m, *_raw_rows(n, m, _sim_transitions, _sim_cost), gamma=0.9,
                         threads=threads)
    _same(h, (ref.row_ptr, ref.col, ref.val, ref.g))
    _same(h, _by_hand(n, m, _sim_transitions, _sim_cost))


def test_from_rows_errors(ingest):
    from paper_2502_14474_gb300 import MDPError
    off, col, prob, g = _raw_rows(60, 3, _sim_transitions, _sim_cost)
    bad = off.copy()
    bad[5] = bad[6] + 1
    with pytest.raises(MDPError, match="BAD_CSR.*offsets decrease at row 5"):
        ingest.from_rows(60, 3, bad, col, prob, g, 0.9)
    c2 = col.copy()
    c2[off[100]] = 60
    c2[off[7]] = -3
    with pytest.raises(MDPError, match=r"successor -3 of \(s, a\) = \(2, 1\)"):
        ingest.from_rows(60, 3, off, c2, prob, g, 0.9, threads=8)
    g2 = g.copy()
    g2[11] = np.inf
    with pytest.raises(MDPError, match=r"NONFINITE.*cost of \(s, a\) = \(3, 2\)"):
        ingest.from_rows(60, 3, off, col, prob, g2, 0.9)
    with pytest.raises(ValueError, match="offsets"):
        ingest.from_rows(60, 3, off[:-1], col, prob, g, 0.9)


def test_from_functions_in_worker_processes(ingest):
    n, m = 60, 3
    ref = ingest.from_functions(n, m, _sim_transitions, _sim_cost, gamma=0.9)
    h = ingest.from_functions(n, m, _sim_transitions, _sim_cost, gamma=0.9, processes=2)
    _same(h, (ref.row_ptr, ref.col, ref.val, ref.g))
    with pytest.raises(RuntimeError, match="state 37"):
        ingest.from_functions(n, m, _sim_fails, _sim_cost, gamma=0.9, processes=2)


def test_pinned_needs_a_device(ingest):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present (the GPU tests cover pinned outputs)")
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        ingest.from_samples(2, 1, [0, 1], [0, 0], [1, 0], None, pinned=True)

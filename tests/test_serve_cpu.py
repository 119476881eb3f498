"""Host logic of the serving loop (queue, admission by memory budget, concurrency)
with a fake solver: no GPU needed."""
import threading
import time

import numpy as np

from paper_2502_14474_gb300 import serve


class _FakeMDP:
    def __init__(self, n):
        self.n, self.m, self.gamma = n, 1, 0.9
        self.row_ptr = np.arange(n + 1, dtype=np.int64)


def _fake_solver(active, peak, lock):
    def solve(req, w):
        with lock:
            active[0] += 1
            peak[0] = max(peak[0], active[0])
        time.sleep(0.01)
        with lock:
            active[0] -= 1
        return np.full(req.mdp.n, req.rid, float), None, {"status": "MDP_OK", "transitions": 1.0}
    return solve


def test_budget_bounds_concurrency_and_fifo_admission():
    active, peak, lock = [0], [0], threading.Lock()
    srv = serve.Server(budget_bytes=300, workers=8, solver=_fake_solver(active, peak, lock),
                       bytes_fn=lambda r: r.mdp.n).start()
    reqs = [serve.Request(rid=i, mdp=_FakeMDP(100)) for i in range(12)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert all(r.status == "MDP_OK" for r in reqs)
    assert peak[0] <= 3 and srv.peak_used <= 300 and srv.peak_active <= 3
    # FIFO: admission times are ordered like the submissions
    t = [r.t_admit for r in reqs]
    assert t == sorted(t)
    assert all(r.V[0] == r.rid for r in reqs)


def test_oversize_request_is_rejected_not_blocking():
    active, peak, lock = [0], [0], threading.Lock()
    srv = serve.Server(budget_bytes=150, workers=2, solver=_fake_solver(active, peak, lock),
                       bytes_fn=lambda r: r.mdp.n).start()
    big = serve.Request(rid=0, mdp=_FakeMDP(1000))
    small = serve.Request(rid=1, mdp=_FakeMDP(100))
    srv.submit(big)
    srv.submit(small)
    srv.close()
    assert big.status == "rejected" and small.status == "MDP_OK"


def test_trace_replay_and_summary():
    active, peak, lock = [0], [0], threading.Lock()
    srv = serve.Server(budget_bytes=1e9, workers=4, solver=_fake_solver(active, peak, lock),
                       bytes_fn=lambda r: r.mdp.n).start()
    arr = serve.poisson_arrivals(40, rate=400.0, seed=5)
    reqs = [serve.Request(rid=i, mdp=_FakeMDP(50), arrival=float(a)) for i, a in enumerate(arr)]
    wall = srv.run_trace(reqs)
    srv.close()
    summ = serve.summarize(reqs, wall)
    assert summ["completed"] == 40 and summ["latency_p99_ms"] >= summ["latency_p50_ms"] > 0
    assert peak[0] >= 2  # arrivals overlapped in service


def test_worker_error_is_isolated():
    def solver(req, w):
        if req.rid == 2:
            raise RuntimeError("poisoned request")
        return np.zeros(1), None, {"status": "MDP_OK", "transitions": 1.0}
    srv = serve.Server(budget_bytes=1e9, workers=2, solver=solver, bytes_fn=lambda r: 1).start()
    reqs = [serve.Request(rid=i, mdp=_FakeMDP(1)) for i in range(5)]
    for r in reqs:
        srv.submit(r)
    srv.close()
    assert [r.status for r in reqs] == ["MDP_OK", "MDP_OK", "error", "MDP_OK", "MDP_OK"]


def test_admission_estimate_follows_the_request_dtypes():
    """A float64 MDP (as the ingest builders return) needs the FP64 remainders on
    the device (4 B per nonzero) and a wider staging copy (4 more per nonzero,
    4 more per cost) than the same MDP in float32."""
    import dataclasses

    import synth
    from paper_2502_14474_gb300 import capi
    m32 = synth.random_sparse(500, 4, 8, 1.0, 0.9, seed=3, dtype=np.float32)
    m64 = dataclasses.replace(m32, val=m32.val.astype(np.float64), g=m32.g.astype(np.float64))
    srv = serve.Server(budget_bytes=1e12, workers=1, solver=lambda r, w: None)
    b32 = srv.request_bytes(serve.Request(rid=0, mdp=m32))
    b64 = srv.request_bytes(serve.Request(rid=1, mdp=m64))
    nnz, rows = m32.nnz, m32.n * m32.m
    assert b64 - b32 == (capi.mdp_bytes_required(m32.n, m32.m, nnz, capi.MDP_F64)
                         - capi.mdp_bytes_required(m32.n, m32.m, nnz, capi.MDP_F32)
                         + 4 * nnz + 4 * rows)
    assert b64 - b32 >= 8 * nnz + 4 * rows
    assert b32 >= capi.mdp_bytes_required(m32.n, m32.m, nnz) + 8 * nnz + 4 * rows


def test_cancel_queued_and_running_requests():
    """cancel() drops a queued request at once and asks a running one to stop;
    the others are served as usual and the budget is released."""
    started = threading.Event()

    def solver(req, w):
        if req.rid == 0:  # a long solve that watches for cancellation
            started.set()
            t0 = time.perf_counter()
            while not req.cancel_requested and time.perf_counter() - t0 < 10:
                time.sleep(0.001)
            return None, None, {"status": "MDP_ERR_CANCELLED" if req.cancel_requested
                                else "MDP_OK", "transitions": 0.0}
        return np.zeros(req.mdp.n), None, {"status": "MDP_OK", "transitions": 1.0}

    srv = serve.Server(budget_bytes=100, workers=1, solver=solver,
                       bytes_fn=lambda r: r.mdp.n).start()
    reqs = [serve.Request(rid=i, mdp=_FakeMDP(60)) for i in range(4)]
    for r in reqs:
        srv.submit(r)
    assert started.wait(5)
    assert srv.cancel(reqs[2])           # still queued: leaves the queue
    assert reqs[2].status == "MDP_ERR_CANCELLED"
    assert srv.cancel(reqs[0])           # running: asked to stop
    srv.close()
    assert [r.status for r in reqs] == ["MDP_ERR_CANCELLED", "MDP_OK",
                                        "MDP_ERR_CANCELLED", "MDP_OK"]
    assert not srv.cancel(reqs[1])       # already finished
    assert srv.used == 0 and srv.active == 0
    summ = serve.summarize(reqs, 1.0)
    assert summ["completed"] == 2 and summ["failed"] == 2


class _PendingCancelHandle:
    """Stands in for a library handle with the C ABI's cancel rule: a cancel
    request made before the solve starts stays pending and the solve returns
    MDP_ERR_CANCELLED at once."""

    def __init__(self, gate, entered):
        self.h = object()
        self.pending = False
        self.gate, self.entered = gate, entered
        self.solved = False

    def solve(self, **kw):
        import torch
        from paper_2502_14474_gb300 import capi
        self.entered.set()
        self.gate.wait(5)          # the test cancels in this window
        if self.pending:
            self.pending = False
            raise capi.MDPError(7, "cancelled before the call started")
        self.solved = True
        return torch.zeros(3), torch.zeros(3, dtype=torch.int32), {"status": "MDP_OK"}

    def close(self):
        pass


def test_cancel_between_publish_and_solve_start_is_not_lost():
    """A cancel() that lands after the worker published the request's handle but
    before the solve's first check reaches the handle and ends the request as
    cancelled (the solve must not run to the end with cancel() having said True)."""
    gate, entered = threading.Event(), threading.Event()
    handles = []

    class Srv(serve.Server):
        def _worker_stream(self):
            return None

        def _open(self, req, stream):
            handles.append(_PendingCancelHandle(gate, entered))
            return handles[-1]

        def _cancel_handle(self, handle):
            for fh in handles:
                if fh.h is handle:
                    fh.pending = True

    srv = Srv(budget_bytes=100, workers=1, bytes_fn=lambda r: 1)
    srv.solver = None
    for w in range(srv.workers):
        t = threading.Thread(target=srv._worker, args=(w,), daemon=True)
        t.start()
        srv.threads.append(t)
    req = serve.Request(rid=0, mdp=_FakeMDP(3))
    srv.submit(req)
    assert entered.wait(5) and req.handle is not None
    assert srv.cancel(req)
    gate.set()
    srv.close()
    assert req.status == "MDP_ERR_CANCELLED", req.status
    assert not handles[0].solved
    assert srv.used == 0 and srv.active == 0

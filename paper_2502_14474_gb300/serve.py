"""Continuous-batching request loop for MDP solves (serving pattern).

Requests (one MDP each, host CSR) arrive over time and wait in a FIFO queue.
The head of the queue is admitted as soon as its device memory
(``mdp_bytes_required``) fits the remaining budget and a worker is free.
Every worker owns a CUDA stream, creates the request's handle from host memory,
runs the inexact policy iteration (the CSR, V and pi stay resident on the GPU
for the whole solve), copies V and pi back, destroys the handle and releases
its memory.  Workers run concurrently (the C ABI calls release the GIL), so
requests that arrive while others are on the GPU join them on the device and
their kernels overlap.  A request's result does not depend on what else runs:
handles share no device state and every reduction has a fixed order.

Latency = completion time - arrival time; the loop reports p50/p99 and
throughput (solves/s).
"""
from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque

import numpy as np

from . import MDP, capi


@dataclasses.dataclass
class Request:
    rid: int
    mdp: object                 # host CSR with n, m, gamma, row_ptr, col, val, g
    arrival: float = 0.0        # seconds since the trace start (scheduled)
    t_arrive: float = 0.0       # wall clock when submitted
    t_admit: float = 0.0
    t_done: float = 0.0
    V: np.ndarray | None = None
    pi: np.ndarray | None = None
    stats: dict | None = None
    status: str = "pending"
    error: str = ""
    nbytes: int = 0
    cancel_requested: bool = False
    handle: int | None = dataclasses.field(default=None, repr=False)  # while solving

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrive


class Server:
    """Admission by device-memory budget, a worker pool of CUDA streams."""

    def __init__(self, budget_bytes: float = 100e9, workers: int = 8, store: str = "f32",
                 solve_opts: dict | None = None, device: int = 0, solver=None,
                 bytes_fn=None):
        """``solver(req, worker_index)`` may replace the GPU solve (it returns
        (V, pi, stats)) and ``bytes_fn(req)`` the device-memory estimate; both
        exist so that the queueing and admission logic can run without a GPU."""
        self.solver = solver
        self.bytes_fn = bytes_fn
        self.budget = int(budget_bytes)
        self.used = 0
        self.workers = workers
        self.store = store
        self.solve_opts = dict(tol=1e-9, inner_rtol=0.1, restart=30)
        if solve_opts:
            self.solve_opts.update(solve_opts)
        self.device = device
        self.cv = threading.Condition()
        self.queue: deque[Request] = deque()
        self.done: list[Request] = []
        self.closed = False
        self.threads = []
        self.peak_used = 0
        self.peak_active = 0
        self.active = 0

    # -- lifecycle -----------------------------------------------------------------
    def start(self):
        if self.solver is None:
            capi.load()
        for w in range(self.workers):
            t = threading.Thread(target=self._worker, args=(w,), daemon=True)
            t.start()
            self.threads.append(t)
        return self

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()

    def request_bytes(self, req: Request) -> int:
        """Device bytes a request holds while admitted: the handle
        (mdp_bytes_required, for the request's probability dtype), the staging
        copy of its host CSR during create (row pointers, columns, values and
        costs at their own widths) and the solve's outputs (float64 V, int32 pi)."""
        if self.bytes_fn is not None:
            return int(self.bytes_fn(req))
        mdp = req.mdp
        nnz, rows = int(mdp.row_ptr[-1]), mdp.n * mdp.m
        vsz, gsz = np.dtype(mdp.val.dtype).itemsize, np.dtype(mdp.g.dtype).itemsize
        b = capi.mdp_bytes_required(mdp.n, mdp.m, nnz,
                                    capi.MDP_F64 if vsz == 8 else capi.MDP_F32,
                                    {"f32": capi.MDP_F32, "bf16": capi.MDP_BF16,
                                     "f16": capi.MDP_F16}[self.store],
                                    self.solve_opts.get("restart", 30))
        staging = (rows + 1) * 8 + nnz * (4 + vsz) + rows * gsz
        return b + staging + mdp.n * 12

    def submit(self, req: Request):
        req.nbytes = self.request_bytes(req)
        if req.nbytes > self.budget:
            req.status = "rejected"
            req.error = "request needs more device memory than the whole budget"
            req.t_arrive = req.t_done = time.perf_counter()
            with self.cv:
                self.done.append(req)
            return
        req.t_arrive = time.perf_counter()
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()

    def cancel(self, req: Request) -> bool:
        """Cancel a request.  A queued one leaves the queue at once with status
        MDP_ERR_CANCELLED; a running one is asked to stop at its solve's next
        host check (mdp_cancel), and ends with that status unless its solve
        finished first.  Returns False when the request had already finished."""
        with self.cv:
            for i, q in enumerate(self.queue):
                if q is req:
                    del self.queue[i]
                    req.cancel_requested = True
                    req.status = "MDP_ERR_CANCELLED"
                    req.t_done = time.perf_counter()
                    self.done.append(req)
                    self.cv.notify_all()
                    return True
            if req.t_done or req.status not in ("pending",):
                return False
            req.cancel_requested = True
            if req.handle is not None:
                self._cancel_handle(req.handle)
            return True

    # -- worker --------------------------------------------------------------------
    def _take(self):
        with self.cv:
            while True:
                if self.queue and self.used + self.queue[0].nbytes <= self.budget:
                    req = self.queue.popleft()
                    self.used += req.nbytes
                    self.active += 1
                    self.peak_used = max(self.peak_used, self.used)
                    self.peak_active = max(self.peak_active, self.active)
                    req.t_admit = time.perf_counter()
                    return req
                if self.closed and not self.queue:
                    return None
                self.cv.wait()

    def _release(self, req):
        with self.cv:
            self.used -= req.nbytes
            self.active -= 1
            self.done.append(req)
            self.cv.notify_all()

    def _worker(self, w):
        if self.solver is not None:
            while True:
                req = self._take()
                if req is None:
                    return
                try:
                    req.V, req.pi, req.stats = self.solver(req, w)
                    req.status = req.stats.get("status", "MDP_OK")
                except Exception as e:
                    req.status = "error"
                    req.error = repr(e)
                req.t_done = time.perf_counter()
                self._release(req)
        stream = self._worker_stream()
        while True:
            req = self._take()
            if req is None:
                return
            try:
                self._serve_one(req, stream)
            except capi.MDPError as e:
                req.status = e.status_name
                req.error = str(e)
            except Exception as e:  # keep serving the other requests
                req.status = "error"
                req.error = repr(e)
            req.t_done = time.perf_counter()
            self._release(req)

    def _worker_stream(self):
        import torch
        torch.cuda.set_device(self.device)
        return torch.cuda.Stream(device=self.device)

    def _open(self, req, stream):
        """The request's handle, created from its host CSR on the worker's stream."""
        return MDP.from_csr(req.mdp, store=self.store, host_input=True,
                            device=f"cuda:{self.device}", stream=stream)

    def _cancel_handle(self, handle):
        capi.mdp_cancel(handle)

    def _serve_one(self, req, stream):
        import contextlib
        import torch
        with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
            h = self._open(req, stream)
            try:
                with self.cv:  # from here on cancel() reaches the solve
                    req.handle = h.h
                    stop = req.cancel_requested
                if stop:
                    raise capi.MDPError(7, "cancelled before the solve started")
                # a cancel() that lands between the lines above and the solve's
                # first check stays pending on the handle, and the library
                # honours it when the solve starts
                V, pi, st = h.solve(raise_on_not_converged=False, **self.solve_opts)
                Vh = V.cpu()
                pih = pi.cpu()
                if stream is not None:
                    stream.synchronize()
            finally:
                with self.cv:
                    req.handle = None
                h.close()
        req.V, req.pi, req.stats = Vh.numpy(), pih.numpy(), st
        req.status = st["status"]

    # -- trace replay ---------------------------------------------------------------
    def run_trace(self, requests, time_scale: float = 1.0):
        """Submit requests at their scheduled arrival times; wait for all of them."""
        t0 = time.perf_counter()
        for req in sorted(requests, key=lambda r: r.arrival):
            delay = t0 + req.arrival * time_scale - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            self.submit(req)
        with self.cv:
            while len(self.done) < len(requests):
                self.cv.wait(timeout=1.0)
        return time.perf_counter() - t0


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def summarize(requests, wall_s: float) -> dict:
    ok = [r for r in requests if r.status == "MDP_OK"]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(1)
    queue = np.array([r.t_admit - r.t_arrive for r in ok]) if ok else np.zeros(1)
    trans = float(sum(r.stats["transitions"] for r in ok))
    return {
        "requests": len(requests),
        "completed": len(ok),
        "failed": len(requests) - len(ok),
        "wall_s": wall_s,
        "solves_per_s": len(ok) / wall_s if wall_s > 0 else 0.0,
        "transitions_per_s": trans / wall_s if wall_s > 0 else 0.0,
        "latency_p50_ms": float(np.percentile(lat, 50) * 1e3),
        "latency_p99_ms": float(np.percentile(lat, 99) * 1e3),
        "latency_max_ms": float(lat.max() * 1e3),
        "queue_p50_ms": float(np.percentile(queue, 50) * 1e3),
        "queue_p99_ms": float(np.percentile(queue, 99) * 1e3),
    }

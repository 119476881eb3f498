#!/usr/bin/env python
"""Throughput of inexact policy iteration on the banded 4M-state MDP.

Workload (seeded, synthetic): n = 2^22 states, m = 8 actions, 16 successors
per (s, a) drawn without replacement from the clipped band [s-4096, s+4096],
Dirichlet(0.5) probabilities (FP32), g ~ U[0,1], gamma = 0.99; 536,870,912
nonzeros (4.3 GB of col+val, larger than the 129 MB L2).

One step = one mdp_solve from V = 0 to a Bellman residual ||TV - V||_inf <= 1e-9
(float-float outer iterate, GMRES(30) inner solves to 0.1 ||TV - V||_inf).
Metric: effective transitions/s = nonzeros touched per second, with every
Bellman sweep counted at nnz and every policy-row SpMV at the policy's nnz.

Prints one JSON line (rank 0).  With --impl reference the FP64 CPU oracle is
timed instead (Bellman sweeps over a bounded sample of the same workload).
Under torchrun each rank solves its own replica (weak scaling, no exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "effective transitions/s (nnz*iters/s)"
UNIT = "transitions/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=None, help="state count override (same recipe)")
    p.add_argument("--tol", type=float, default=1e-9)
    p.add_argument("--restart", type=int, default=30)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--profile-bellman", type=int, default=0,
                   help="only run N float-float Bellman backups (for ncu captures)")
    p.add_argument("--fp-rates", action="store_true",
                   help="time dense FP64 and FP32 (no TF32) matrix products through torch "
                        "(cuBLAS) and print the achieved rates: the measured basis for doing "
                        "the high-precision arithmetic in float-float on the FP32 pipes")
    p.add_argument("--profile-solve", action="store_true",
                   help="one solve, nothing else (for ncu launch lists)")
    p.add_argument("--no-profile", action="store_true",
                   help="no per-kernel events in the timed region (roofline omitted)")
    p.add_argument("--workload", choices=["banded4m", "grid4096", "batch512", "serve"],
                   default="banded4m",
                   help="banded4m: the headline MDP; grid4096: the 4096^2 grid world of the "
                        "precision path (gamma = 0.999); batch512: 512 uneven random MDPs "
                        "solved concurrently; serve: Poisson request stream through the "
                        "continuous-batching loop")
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--batch-mode", choices=["fused", "streams"], default="fused",
                   help="batch512: every solve phase of all MDPs in one launch (fused), or "
                        "concurrent handles on a pool of streams")
    p.add_argument("--streams", type=int, default=16)
    p.add_argument("--requests", type=int, default=10000)
    p.add_argument("--pool", type=int, default=512,
                   help="serve: distinct MDPs drawn from the uneven-batch distribution")
    p.add_argument("--saturation-rate", type=float, default=2000.0)
    p.add_argument("--saturation-requests", type=int, default=3000)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--budget-gb", type=float, default=100.0)
    p.add_argument("--store", choices=["f32", "bf16", "f16"], default="f32",
                   help="probabilities of the inner GMRES SpMV")
    p.add_argument("--inner-norm", choices=["2", "inf"], default="2")
    p.add_argument("--inner", choices=["gmres", "richardson", "bicgstab"], default="gmres",
                   help="inner solver of the evaluation step: GMRES (iPI), Richardson "
                        "sweeps (modified policy iteration; with --max-inner 1 it is value "
                        "iteration) or BiCGStab")
    p.add_argument("--s-step", type=int, default=None,
                   help="GMRES block size (0 = classical Arnoldi; default: the library's)")
    p.add_argument("--max-inner", type=int, default=None,
                   help="cap on GMRES steps per outer iteration (default 10000; 100 for "
                        "grid4096, whose early policies make the evaluation nearly singular)")
    return p.parse_args()


def aggregate(ms_local: float, transitions_local: float, dist=None, device=None):
    """Whole-job throughput of weak-scaled replicas: every rank solved its own
    copy; the job time is the slowest rank's, the work is the sum over ranks.
    Returns (ms_max, value_transitions_per_s)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, transitions_local / (ms_local / 1e3)
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    w = torch.tensor([transitions_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    ms_max = float(t.item())
    return ms_max, float(w.item()) / (ms_max / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _traffic_record(kernel, n):
    """DRAM bytes per launch of `kernel` from the committed ncu record, or None when
    the record is for another kernel or size, or the kernel's sources changed."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    try:
        rec = {}
        for line in open(path):
            line = line.strip()
            if line and not line.startswith("#") and "=" in line:
                k, v = line.split("=", 1)
                rec[k.strip()] = v.strip()
        if rec.get("kernel") != kernel or int(rec.get("scaled_n", -1)) != n:
            return None
        h = hashlib.sha256()
        for f in rec["sources"].split():
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != rec.get("sources_sha256"):
            return None
        return float(rec["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


WORKLOAD = "banded4m"


def _bellman_latency(h, host, stream, dev, reps=50):
    """p50/p99 over `reps` single FP32 Bellman backups (K1) through mdp_bellman, with
    CUDA events on the solve stream around each call, and the achieved GB/s of the
    median against K1's algorithmic bytes (nnz*(4 col + 4 val) + rows*4 g (+ row
    pointers when rows differ in length) + n*(4 V + 4 V' + 4 pi))."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    V = torch.rand(host.n, dtype=torch.float32, device=dev, generator=gen) * 50.0
    lens = np.diff(host.row_ptr)
    rp_bytes = 0 if lens.min() == lens.max() else (len(host.row_ptr)) * 4
    nbytes = host.nnz * 8 + host.n * host.m * 4 + rp_bytes + host.n * 12
    ms = []
    with torch.cuda.stream(stream):
        for i in range(reps + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.bellman(V, want_v=True, want_pi=True, want_r=False)
            b.record(stream)
            b.synchronize()
            if i >= 3:
                ms.append(a.elapsed_time(b))
    p50, p99 = float(np.percentile(ms, 50)), float(np.percentile(ms, 99))
    return {"kernel": "bellman_f32 (K1)", "reps": reps, "p50_ms": p50, "p99_ms": p99,
            "bytes": float(nbytes), "GBps_p50": nbytes / (p50 / 1e3) / 1e9}


def _workload(n=None, s0=0, s1=None):
    import synth
    if WORKLOAD == "grid4096":
        side = int(round(n ** 0.5)) if n else None
        return synth.grid_4096(s0=s0, s1=s1, side=side)
    return synth.banded_4m(n=n, s0=s0, s1=s1)


def _cpu_sample_bellman(n, seconds, s1=1 << 18):
    """Time the FP64 oracle's Bellman sweep on states [0, s1) of the workload."""
    import oracle
    blk = _workload(n=n, s0=0, s1=min(s1, n if n else 1 << 22))
    V = np.random.default_rng(0).random(blk.n) * 100
    oracle.bellman(blk, V)  # load + warm
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.bellman(blk, V)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    return dict(value=blk.nnz * reps / el, unit=UNIT, cores=int(omp) if omp else cores,
                kind="oracle",
                sample=(f"FP64 oracle Bellman sweep (T V with greedy argmin) over states "
                        f"[0, {blk.n_local}) of the workload ({blk.nnz} nnz), {reps} sweeps, "
                        f"{el:.1f} s"))


def _oracle_error_blocks(n_total, V, pi, tol, block=4096):
    """The FP64 oracle's certificate of a GPU result on three sampled blocks of
    states (both ends of the state range and one in the middle), run on the host
    after the timed region: ||T V - V||_inf in FP64 over the blocks, the bound
    ||V - V*||_inf <= res / (1 - gamma) it implies for the whole vector when the
    whole residual is that small, and the greedy actions that differ from the
    oracle's on states whose oracle Q-gap exceeds 2 tol."""
    import oracle
    res, mism, checked, gamma = 0.0, 0, 0, None
    starts = (0, n_total // 3, max(0, n_total - block))
    for s0 in starts:
        s1 = min(n_total, s0 + block)
        blk = _workload(n=n_total, s0=s0, s1=s1)
        cert = oracle.certificate(blk, V)
        gamma = float(blk.gamma)
        res = max(res, cert["res_inf"])
        clear = cert["gap"] > 2 * tol + 1e-12
        mism += int(np.count_nonzero(pi[s0:s1][clear] != cert["pi"][clear]))
        checked += s1 - s0
    vmax = float(np.max(np.abs(V))) if len(V) else 0.0
    bound = res / (1.0 - gamma)
    return {"kind": "FP64 oracle certificate on sampled blocks",
            "blocks": [[s0, min(n_total, s0 + block)] for s0 in starts],
            "states_checked": checked, "res_inf_fp64": res, "bound_inf": bound,
            "bound_rel": bound / vmax if vmax > 0 else None,
            "pi_mismatch_on_clear_gap": mism}


def _oracle_error_whole(items, tol):
    """The FP64 oracle's certificate of whole GPU results (small MDPs): the largest
    ||T V - V||_inf, the largest bound res / (1 - gamma) on ||V - V*||_inf, and the
    greedy actions that differ from the oracle's on clear-gap states.  ``items``
    holds (mdp, V, pi) triples."""
    import oracle
    res, bound, mism, states = 0.0, 0.0, 0, 0
    for mdp, V, pi in items:
        cert = oracle.certificate(mdp, V)
        res = max(res, cert["res_inf"])
        bound = max(bound, cert["bound"])
        clear = cert["gap"] > 2 * tol + 1e-12
        mism += int(np.count_nonzero(np.asarray(pi)[clear] != cert["pi"][clear]))
        states += mdp.n
    return {"kind": "FP64 oracle certificate of whole solves", "solves": len(items),
            "states_checked": states, "res_inf_fp64": res, "bound_inf": bound,
            "pi_mismatch_on_clear_gap": mism}


def _timed_oracle(fn):
    """Run fn() and return (result, seconds, host threads available)."""
    t0 = time.perf_counter()
    r = fn()
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    return r, el, int(omp) if omp else cores


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    n = args.n
    blk = _workload(n=n, s0=0, s1=min(1 << 18, n if n else 1 << 22))
    V = np.random.default_rng(0).random(blk.n) * 100
    for _ in range(max(args.warmup, 0)):
        oracle.bellman(blk, V)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        TV, _ = oracle.bellman(blk, V)
    el = time.perf_counter() - t0
    value = blk.nnz * args.steps / el
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"FP64 oracle Bellman sweep over states [0, {blk.n_local}) of the banded "
              f"workload ({blk.nnz} nnz) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": blk.name, "n_states": 1 << 22 if n is None else n, "m": 8,
                       "successors": 16, "band": 4096, "gamma": 0.99, "seed": 2,
                       "sample_states": blk.n_local},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """512 independent random MDPs of uneven size solved concurrently (one JSON line)."""
    import torch
    import synth
    from paper_2502_14474_gb300 import MDP, capi
    t0 = time.perf_counter()
    params = synth.uneven_batch_params(args.batch_count, seed=4)
    mdps = [synth.uneven_mdp(p) for p in params]
    gen_s = time.perf_counter() - t0
    hs = [MDP.from_csr(m, autotune=True) for m in mdps]
    nnz = sum(m.nnz for m in mdps)
    Vs = [torch.empty(m.n, dtype=torch.float64, device="cuda") for m in mdps]
    pis = [torch.empty(m.n, dtype=torch.int32, device="cuda") for m in mdps]
    opts = capi.mdp_default_opts()
    opts.max_inner = args.max_inner

    fstream = torch.cuda.Stream()

    def go(streams, mode=None):
        mode = mode or args.batch_mode
        torch.cuda.synchronize()
        t = time.perf_counter()
        if mode == "fused":
            stats, status = capi.mdp_batch_solve_fused([h.h for h in hs], Vs, pis, opts=opts,
                                                       stream=fstream, raise_on_error=False)
        else:
            stats, status = capi.mdp_batch_solve([h.h for h in hs], Vs, pis, opts=opts,
                                                 n_streams=streams, raise_on_error=False)
        torch.cuda.synchronize()
        return time.perf_counter() - t, stats, status

    if args.profile_solve:  # one batch solve, nothing else (for ncu launch lists)
        el, stats, _ = go(args.streams)
        print(json.dumps({"profile_batch_ms": el * 1e3,
                          "policy_sweeps": sum(st["policy_sweeps"] for st in stats)}))
        return 0
    for _ in range(max(1, args.warmup)):
        go(args.streams)
    times, stats, status = [], None, None
    for _ in range(args.steps):
        el, stats, status = go(args.streams)
        times.append(el)
    other = "streams" if args.batch_mode == "fused" else "fused"
    other_el = min(go(args.streams, other)[0] for _ in range(2))
    seq_el, _, _ = go(1, "streams")
    trans = sum(st["transitions"] for st in stats)
    el = float(np.median(times))
    sample = list(range(0, len(mdps), 100))
    res = [stats[i]["residual_inf"] for i in sample]
    # CPU leg, after the timed runs: the FP64 oracle certifies the 1% sample of
    # results (every 100th MDP) and is timed on Bellman sweeps over the same MDPs
    oracle_error = cpu = None
    if not args.no_cpu_baseline:
        import oracle
        items = [(mdps[i], Vs[i].cpu().numpy(), pis[i].cpu().numpy()) for i in sample]
        oracle_error = _oracle_error_whole(items, 1e-9)

        def sweeps():
            reps, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < args.cpu_seconds:
                for mdp, V, _ in items:
                    oracle.bellman(mdp, V)
                reps += 1
            return reps
        reps, cpu_s, cores = _timed_oracle(sweeps)
        cnnz = sum(mdp.nnz for mdp, _, _ in items)
        cpu = {"value": cnnz * reps / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": (f"FP64 oracle Bellman sweeps over the {len(items)} sampled MDPs "
                          f"({cnnz} nnz), {reps} rounds, {cpu_s:.1f} s")}
    line = {"metric": METRIC, "value": trans / el, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"uneven_batch_{len(mdps)}", "mdps": len(mdps), "nnz": nnz,
                       "n_range": [min(m.n for m in mdps), max(m.n for m in mdps)],
                       "mode": args.batch_mode, "streams": args.streams, "tol": 1e-9,
                       "autotune": True, "generation_s": gen_s},
            f"{other}_ms": other_el * 1e3,
            "converged": sum(1 for x in status if x == "MDP_OK"),
            "sequential_ms": seq_el * 1e3, "speedup_vs_one_stream": seq_el / el,
            "solve_residual_sample": res, "oracle_error": oracle_error, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    for h in hs:
        h.close()
    return 0


def run_serve(args):
    """Poisson request stream through the continuous-batching loop (one JSON line).

    Requests are drawn from the uneven-batch distribution (n log-uniform in
    [2e3, 2e5], m in {2..16}, 4..32 successors per row, gamma in [0.9, 0.999]):
    a pool of ``--pool`` independent draws (distinct seeds), plus 1% large
    requests (n = 2^20, m = 8, 16 successors) from four distinct large MDPs.
    The trace runs at the offered rate, then a shorter trace at
    ``--saturation-rate`` measures the loop's throughput and latency when it
    cannot keep up."""
    import torch
    import synth
    from paper_2502_14474_gb300 import serve
    t0 = time.perf_counter()
    rng = np.random.default_rng(5)
    pool = [synth.uneven_mdp(p) for p in synth.uneven_batch_params(args.pool, seed=5)]
    large = [synth.random_sparse(1 << 20, 8, 16, 1.0, 0.99, seed=5_000_000 + i,
                                 dtype=np.float32, name="random_n1048576_m8_k16")
             for i in range(4)]
    # request payloads live in pinned host memory (as a front end that receives
    # them into registered buffers would hold them): host-to-device copies are
    # then asynchronous DMA instead of staged pageable copies
    for mdp in pool + large:
        for k in ("row_ptr", "col", "val", "g"):
            setattr(mdp, k, torch.from_numpy(getattr(mdp, k)).pin_memory().numpy())
    gen_s = time.perf_counter() - t0

    def trace(count, rate, seed, rid0):
        arrivals = serve.poisson_arrivals(count, rate, seed=seed)
        out = []
        for i, a in enumerate(arrivals):
            if rng.random() < 0.01:
                mdp = large[int(rng.integers(len(large)))]
            else:
                mdp = pool[int(rng.integers(len(pool)))]
            out.append(serve.Request(rid=rid0 + i, mdp=mdp, arrival=float(a)))
        return out

    srv = serve.Server(budget_bytes=args.budget_gb * 1e9, workers=args.streams,
                       solve_opts={"max_inner": args.max_inner}).start()
    # warm the library, the kernels of both request classes and the memory pool
    # on a few requests outside the trace (a server warms up before it takes traffic)
    warm = [serve.Request(rid=-1 - i, mdp=m) for i, m in enumerate(pool[:4] + large[:1])]
    for r in warm:
        srv.submit(r)
    with srv.cv:
        while len(srv.done) < len(warm):
            srv.cv.wait(timeout=1.0)
        srv.done.clear()
    reqs = trace(args.requests, args.rate, 5, 0)
    wall = srv.run_trace(reqs)
    summ = serve.summarize(reqs, wall)
    peak_active, peak_used = srv.peak_active, srv.peak_used
    sat = None
    if args.saturation_requests > 0:
        with srv.cv:
            srv.done.clear()
        sreqs = trace(args.saturation_requests, args.saturation_rate, 6, 10**7)
        swall = srv.run_trace(sreqs)
        sat = serve.summarize(sreqs, swall)
        sat["offered_rate_per_s"] = args.saturation_rate
    srv.close()
    # 1% of the requests: the float-float Bellman residual their solves end on,
    # and (CPU leg, after the traces) the FP64 oracle's certificate of their results
    sample = [r for r in reqs if r.rid % 100 == 0 and r.status == "MDP_OK"]
    oracle_error = None
    if not args.no_cpu_baseline:
        oracle_error, cpu_s, cores = _timed_oracle(
            lambda: _oracle_error_whole([(r.mdp, r.V, r.pi) for r in sample], 1e-9))
        oracle_error["oracle_s"] = cpu_s
        oracle_error["cores"] = cores
    line = {"metric": "solves/s (with p50/p99 latency)", "value": summ["solves_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "poisson_request_stream", "requests": args.requests,
                       "rate_per_s": args.rate, "budget_gb": args.budget_gb,
                       "workers": args.streams, "pool_mdps": len(pool),
                       "pool": "independent draws of the uneven-batch distribution",
                       "large_fraction": 0.01, "large_mdps": len(large),
                       "large": "n=2^20, m=8, 16 successors", "generation_s": gen_s},
            "serving": summ, "saturation": sat, "peak_active": peak_active,
            "peak_budget_gb": peak_used / 1e9,
            "residual_sample": {"requests": len(sample),
                                "max_residual_inf": max((r.stats["residual_inf"] for r in sample),
                                                        default=None)},
            "oracle_error": oracle_error}
    print(json.dumps(line), flush=True)
    return 0


def run_fp_rates():
    """Achieved dense FP64 and FP32 (CUDA-core) FMA rates of this GPU, from cuBLAS
    GEMMs of 8192^3 (2 N^3 flops each), best of 5 after 2 warm-ups, CUDA events."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        n = 8192
        a = torch.rand(n, n, dtype=dt, device="cuda")
        b = torch.rand(n, n, dtype=dt, device="cuda")
        best = None
        for it in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.mm(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            if it >= 2:
                best = ms if best is None else min(best, ms)
        out[name + "_tflops"] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b
    out["fp32_over_fp64"] = out["fp32_tflops"] / out["fp64_tflops"]
    print(json.dumps({"fp_rates": out, "how": "torch.mm 8192^3, TF32 off, best of 5"}))
    return 0


def main():
    global WORKLOAD
    args = _args()
    WORKLOAD = args.workload
    if args.fp_rates:
        return run_fp_rates()
    if args.max_inner is None:
        args.max_inner = 100 if args.workload == "grid4096" else 10000
    if args.workload == "batch512":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_2502_14474_gb300 import MDP, capi

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    host = _workload(n=args.n)
    nnz = host.nnz
    dev = torch.device("cuda", local)
    # a dedicated stream: the library replays each GMRES restart cycle as a CUDA
    # graph there (the legacy default stream cannot be captured)
    solve_stream = torch.cuda.Stream(device=dev)
    h = MDP.from_csr(host, store=args.store, stream=solve_stream)
    opts = dict(tol=args.tol, inner_rtol=0.1, restart=args.restart, inner_norm=args.inner_norm,
                max_inner=args.max_inner, inner=args.inner, max_outer=100000, s_step=args.s_step)

    if args.profile_bellman:
        V = torch.zeros(host.n, dtype=torch.float64, device=dev)
        for _ in range(args.profile_bellman):
            out = h.bellman(V, want_v=True, want_pi=True, want_r=True)
            V = out["V"]
        torch.cuda.synchronize()
        print(json.dumps({"profile_bellman": args.profile_bellman, "res_inf": out["res_inf"]}))
        return 0
    if args.profile_solve:
        _, _, st = h.solve(**opts)
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve": st}))
        return 0

    # ---- warm-up -------------------------------------------------------------
    for _ in range(args.warmup):
        V, pi, st = h.solve(**opts)
    torch.cuda.synchronize()

    # ---- timed region: K full solves (no per-launch events) ---------------------
    stream = solve_stream
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]
                           if ws == 1 else local)

    def timed(profile: bool):
        h.profile(profile)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        # an event between consecutive solves as well: the per-solve times give
        # the median and spread of the step (events cost nothing inside a solve)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        out = []
        for i in range(args.steps):
            V_last, pi_last, st_ = h.solve(**opts)
            out.append(st_)
            last[:] = [V_last, pi_last]
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        elapsed = ev[0].elapsed_time(ev[-1])
        step_ms[:] = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        prof_ = h.profile_read()
        h.profile(False)
        return elapsed, out, prof_

    last = []
    step_ms = []
    sampler.start()
    time.sleep(0.3)
    ms, stats, prof_plain = timed(False)
    steps_plain = list(step_ms)
    V_res = last[0].cpu().numpy()
    pi_res = last[1].cpu().numpy()
    clocks = sampler.stop()
    trans = sum(s["transitions"] for s in stats)
    ms_max, value = aggregate(ms, trans, dist if ws > 1 else None, dev)
    # ---- second timed region, same K solves, CUDA events around every launch on
    # the solve stream: per-kernel durations for the roofline (the events add ~7%
    # to a step, so they are kept out of the headline region)
    prof = None
    if not args.no_profile:
        _, _, prof = timed(True)
    else:
        prof = prof_plain

    # ---- roofline of the dominant kernel (largest event-timed total) ----------
    kinds = prof["kinds"]
    dom = max(kinds, key=lambda k: kinds[k]["ms"])
    dk = kinds[dom]
    peak, peak_src = _peaks()
    achieved = (dk["bytes"] / dk["launches"]) / (dk["ms"] / dk["launches"] / 1e3) / 1e9 \
        if dk["launches"] else 0.0
    traffic = _traffic_record(dom, host.n)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "bytes_per_launch": dk["bytes"] / max(1, dk["launches"]),
                "ms_per_launch": dk["ms"] / max(1, dk["launches"]),
                "launches": dk["launches"]} if not args.no_profile else None
    per_kernel = {k: {"launches": v["launches"], "skipped": v["skipped"],
                      "ms_total": round(v["ms"], 3),
                      "p50_ms": round(v["p50_ms"], 4), "p99_ms": round(v["p99_ms"], 4),
                      "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 and v["bytes"]
                      else None}
                  for k, v in kinds.items() if v["launches"] or v["skipped"]}

    # ---- per-call latency of the FP32 Bellman backup (the K1 kernel) -----------
    bellman_k1 = None if args.no_profile else _bellman_latency(h, host, stream, dev)

    # ---- end to end through the public API with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()
        hp = {k: pin(getattr(host, k)) for k in ("row_ptr", "col", "val", "g")}
        Vh = torch.empty(host.n, dtype=torch.float64).pin_memory()
        pih = torch.empty(host.n, dtype=torch.int32).pin_memory()
        h.close()
        h = None
        torch.cuda.empty_cache()
        h2d = sum(x.numel() * x.element_size() for x in hp.values())
        d2h = Vh.numel() * 8 + pih.numel() * 4
        e2e_steps = max(1, min(args.steps, 3))

        def one():
            m = MDP(host.n, host.m, hp["row_ptr"].numpy(), hp["col"].numpy(), hp["val"].numpy(),
                    hp["g"].numpy(), host.gamma, store=args.store, stream=solve_stream)
            Vd, pid, s = m.solve(**opts)
            Vh.copy_(Vd, non_blocking=True)
            pih.copy_(pid, non_blocking=True)
            torch.cuda.synchronize()
            m.close()
            return s
        one()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        tr = 0.0
        for _ in range(e2e_steps):
            tr += one()["transitions"]
        el = time.perf_counter() - t0
        te = torch.tensor([el], dtype=torch.float64, device=dev)
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": tr * ws / float(te.item()), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "ms_per_step": float(te.item()) / e2e_steps * 1e3}
    if h is not None:
        h.close()

    # ---- CPU leg: the FP64 oracle timed on the host, and its certificate of the
    # result of the last timed solve (after the timed regions)
    cpu, oracle_error = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = _cpu_sample_bellman(args.n, args.cpu_seconds)
        oracle_error = _oracle_error_blocks(host.n, V_res, pi_res, args.tol)

    if rank == 0:
        st0 = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "step_ms": {"each": [round(x, 3) for x in steps_plain],
                        "median": statistics.median(steps_plain),
                        "min": min(steps_plain), "max": max(steps_plain)},
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": host.name, "n_states": host.n, "m": host.m, "nnz": nnz,
                       "gamma": host.gamma, "seed": 2 if args.workload == "banded4m" else 3,
                       "tol": args.tol,
                       "s_step": (args.s_step if args.s_step is not None
                                  else capi.mdp_default_opts().s_step),
                       "inner": (f"gmres({args.restart})" if args.inner == "gmres"
                                 else "bicgstab" if args.inner == "bicgstab"
                                 else ("value iteration" if args.max_inner == 1
                                       else "richardson (modified PI)")),
                       "eta": 0.1,
                       "inner_norm": args.inner_norm, "max_inner": args.max_inner,
                       "inner_probabilities": args.store,
                       "outer_iterate": "float-float (hi+lo FP32)", "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{ws}"},
            "time_to_tol_s": ms_max / args.steps / 1e3,
            "solve": {"outer_iters": st0["outer_iters"], "inner_iters": st0["inner_iters"],
                      "bellman_sweeps": st0["bellman_sweeps"],
                      "policy_sweeps": st0["policy_sweeps"],
                      "residual_inf": st0["residual_inf"],
                      "transitions_per_solve": st0["transitions"],
                      "residual_history": st0["residual_history"],
                      "inner_history": st0["inner_history"]},
            "roofline": roofline,
            "kernels": per_kernel,
            "bellman_k1": bellman_k1,
            "gpu_launches": prof_plain["total_launches"],
            "roofline_region": "second timed pass of the same solves with CUDA events around "
                               "every launch on the solve stream",
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "oracle_error": oracle_error,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

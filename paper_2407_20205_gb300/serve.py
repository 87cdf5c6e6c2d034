"""Replay a stream of permanent requests against the serving C API.

    python -m paper_2407_20205_gb300.serve --jobs 5000 --nmax 32 --rho 0.7

The trace is the serving mix: n uniform in [nmin, nmax]; 80% uniform
entries, 15% sparse (P(0) = 0.6), 5% known-answer matrices (permuted
identities, J_n, block-diagonal products under monomial transforms).
Arrivals are Poisson with rate rho * C / E[2^n], C the GPU's measured
capacity in subsets/s, so rho is the offered load.  Latency is the time from
a request's scheduled arrival to its result becoming visible on the host.
The same trace is also served FIFO with one matrix per launch (perm_f3 per
request, in arrival order) as the baseline.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding, inputs


def make_trace(seed: int, jobs: int, nmin: int, nmax: int):
    return [inputs.serve_job(seed, j, nmin, nmax) for j in range(jobs)]


def _bands(nmin, nmax):
    edges = [(12, 24), (25, 32), (33, 40), (41, 64)]
    out = [(max(a, nmin), min(b, nmax)) for a, b in edges if a <= nmax and b >= nmin]
    if nmin < 12:
        out = [(nmin, 11)] + out
    return out


def latency_stats(ns, lat_s, nmin, nmax):
    lat = np.asarray(lat_s)
    ns = np.asarray(ns)
    res = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}
    bands = {}
    for a, b in _bands(nmin, nmax):
        m = (ns >= a) & (ns <= b)
        if m.any():
            bands[f"{a}-{b}"] = {"jobs": int(m.sum()), "p50_ms": float(np.percentile(lat[m], 50) * 1e3),
                                 "p99_ms": float(np.percentile(lat[m], 99) * 1e3)}
    res["bands"] = bands
    return res


def replay(trace, arrivals, cfg_overrides=None):
    """Serve the trace through a pf3 context; returns results, latencies and
    throughput over the makespan."""
    cfg_overrides = cfg_overrides or {}
    with binding.ServeContext(**cfg_overrides) as ctx:
        # warm the path once (untimed)
        t = ctx.submit(np.eye(13, dtype=np.uint8))
        ctx.wait(t)
        tickets = []
        t0 = binding.now_ns()
        sched = [t0 + int(a * 1e9) for a in arrivals]
        for (n, kind, A, parts), ts in zip(trace, sched):
            while binding.now_ns() < ts:
                pass
            while True:
                tk = ctx.try_submit(A)
                if tk != binding.PF3_EBUSY:
                    break
                time.sleep(50e-6)
            if tk < 0:
                raise binding.PF3Error(tk, "perm_f3_submit")
            tickets.append(tk)
        results = [ctx.wait(tk) for tk in tickets]
        done = [ctx.times(tk)[1] for tk in tickets]
        stats = ctx.stats()
    lat = [(d - s) * 1e-9 for d, s in zip(done, sched)]
    makespan = (max(done) - t0) * 1e-9
    return results, lat, makespan, stats


def replay_fifo(trace, arrivals):
    """Baseline: one matrix per launch, in arrival order, on the calling thread."""
    results, lat = [], []
    t0 = binding.now_ns()
    sched = [t0 + int(a * 1e9) for a in arrivals]
    for (n, kind, A, parts), ts in zip(trace, sched):
        while binding.now_ns() < ts:
            pass
        results.append(binding.perm_f3(A))
        lat.append((binding.now_ns() - ts) * 1e-9)
    makespan = (binding.now_ns() - t0) * 1e-9
    return results, lat, makespan


def measure_capacity(n: int = 36, reps: int = 3) -> float:
    """Gray subsets per second of the single-matrix walk on this GPU: the
    best of `reps` full walks of the seeded uniform n x n matrix, after one
    warm-up (a 36 x 36 walk takes about 9 ms on a GB300)."""
    A = inputs.uniform_matrix(n, n)
    binding.perm_f3(A)
    best = float("inf")
    for _ in range(reps):
        t = time.perf_counter()
        binding.perm_f3(A)
        best = min(best, time.perf_counter() - t)
    return float(1 << n) / best


def run(jobs=5000, nmin=12, nmax=32, rho=0.7, seed=inputs.SEED_SERVE, capacity=None, fifo=True,
        cfg_overrides=None):
    trace = make_trace(seed, jobs, nmin, nmax)
    ns = [t[0] for t in trace]
    work = float(sum(1 << n for n in ns))
    mean_work = float(np.mean([(1 << n) for n in range(nmin, nmax + 1)]))
    if capacity is None:
        capacity = measure_capacity()
    rate = rho * capacity / mean_work
    arrivals = inputs.poisson_arrivals(seed, jobs, rate)
    res, lat, makespan, stats = replay(trace, arrivals, cfg_overrides)
    out = {"jobs": jobs, "n_range": [nmin, nmax], "rho": rho, "rate_per_s": rate,
           "capacity_subsets_per_s": capacity, "total_subsets": work,
           "batched": {"makespan_s": makespan, "jobs_per_s": jobs / makespan, "subsets_per_s": work / makespan,
                       **latency_stats(ns, lat, nmin, nmax), **stats}}
    if fifo:
        fres, flat, fmk = replay_fifo(trace, arrivals)
        out["fifo_one_per_launch"] = {"makespan_s": fmk, "jobs_per_s": jobs / fmk, "subsets_per_s": work / fmk,
                                      **latency_stats(ns, flat, nmin, nmax)}
        out["results_identical"] = bool(fres == res)
    return out, res, trace


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=5000)
    ap.add_argument("--nmin", type=int, default=12)
    ap.add_argument("--nmax", type=int, default=32)
    ap.add_argument("--rho", type=float, default=0.7)
    ap.add_argument("--capacity", type=float, default=None,
                    help="subsets/s the offered load is scaled to (default: measured on a 36x36 walk)")
    ap.add_argument("--no-fifo", action="store_true")
    ap.add_argument("--small-work-log2", type=int, default=None,
                    help="requests with at most 2^k Gray indices left go first (default 33)")
    ap.add_argument("--chunk-log2", type=int, default=None)
    ap.add_argument("--launch-budget-log2", type=int, default=None)
    a = ap.parse_args()
    cfg = {}
    if a.small_work_log2 is not None:
        cfg["small_work_log2"] = a.small_work_log2
    if a.chunk_log2 is not None:
        cfg["chunk_log2"] = a.chunk_log2
    if a.launch_budget_log2 is not None:
        cfg["launch_budget"] = 1 << a.launch_budget_log2
    out, _, _ = run(a.jobs, a.nmin, a.nmax, a.rho, capacity=a.capacity, fifo=not a.no_fifo, cfg_overrides=cfg)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

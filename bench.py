#!/usr/bin/env python3
"""Benchmark: Gray-code Ryser subsets/s for perm(A) mod 3 on one GB300.

Workload (one "step"): the permanent of the seeded uniform 36 x 36 matrix and
of the seeded uniform 40 x 40 matrix, each a full walk of all 2^n Gray
indices in its own launch (one matrix per launch).  value = subsets/s
(2^36 + 2^40 per step) with the matrices resident in HBM; e2e = the same
through the host-pointer C entry point perm_f3 (input copied in, result
copied out, every call).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-batch] [--no-cpu-baseline] [--no-serve] [--serve-jobs J]
                  [--no-config1] [--no-long]

Secondary measurements go under "extra": the seeded 20 x 20 matrix (one
launch per permanent), the batched Monte Carlo workload (200,000 seeded
24 x 24 matrices in one call, against the same matrices one launch each), the
serving mix (Poisson arrivals, n in 12..40, against FIFO one matrix per
launch) and the seeded 48 x 48 matrix (all 2^48 Gray indices in bounded
launches).

With N > 1 (torchrun, one rank per GPU) every rank walks its 1/N share of each
matrix's Gray range (Sec. 3.1's block split) and the two 64-bit counts are
summed across ranks at the end of each step (strong scaling).

--impl reference times the CPU oracle (the plain integer Ryser walk) on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F3 Ryser Gray-code subsets/sec on 1 GB300; batched perms/sec; p50/p99 latency"
UNIT = "subsets/s"
SIZES = (36, 40)
def i_alg(G: int) -> float:
    """Minimal ALU-pipe instructions per subset of the grouped walk.  Per group
    of 2^G Gray indices: one row step on the low word of the base (3 LOP3),
    the base's zero test (1), and 2^G - 1 probes.  A probe needs two LOP3 (the
    function "column of v + c is nonzero" has four inputs); the second LOP3
    can also write its zero test as a predicate, and one three-input predicate
    OR folds two such tests into the group's running flag, so a probe costs at
    least 2.5 instructions.  The compiled kernel executes a little more (see
    profiles/walk_single_n36.md)."""
    return (3 + 1 + 2.5 * ((1 << G) - 1)) / (1 << G)


KERNEL_FILES = {"single": ("pf3_device.cuh", "pf3_internal.h", "pf3_single.cu"),
                "batch": ("pf3_device.cuh", "pf3_internal.h", "pf3_batch.h", "pf3_batch.cu")}


def kernel_source_hash(kind: str = "single") -> str:
    """Hash of the sources a kernel is compiled from: ties a committed ncu
    summary to the kernel it measured."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2407_20205_gb300", "csrc")
    for name in KERNEL_FILES[kind]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def profiled(summary="walk_single_n36.md", kind="single"):
    """Figures from the committed ncu summary of a walk kernel (DRAM bytes per
    launch, executed ALU instructions per subset, ALU pipe busy), or {} when
    the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except OSError:
        return {}
    vals = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-* ")
        if ":" in line and line.startswith(("source_hash", "dram_bytes_per_launch", "alu_inst_per_subset",
                                            "alu_pipe_busy")):
            k, v = line.split(":", 1)
            vals[k.strip(" `")] = v.strip(" `")
    if vals.get("source_hash") != kernel_source_hash(kind):
        return {}
    out = {}
    for k in ("dram_bytes_per_launch", "alu_inst_per_subset", "alu_pipe_busy"):
        try:
            out[k] = float(vals[k])
        except (KeyError, ValueError):
            pass
    return out


def profiled_traffic(summary="walk_single_n36.md"):
    return profiled(summary).get("dram_bytes_per_launch")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def matrices():
    from paper_2407_20205_gb300 import inputs
    seeds = {36: inputs.SEED_N36, 40: inputs.SEED_N40}
    return {n: inputs.uniform_matrix(seeds[n], n) for n in SIZES}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="pf3_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out.update({"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                    "reasons": sorted(reasons), "samples": len(rows)})
        return out


def cpu_sample(A, seconds_target=12.0, max_log2=34):
    """Time the oracle's Gray walk on a bounded sub-range of A's index space,
    on all host cores; grow the range until it takes ~seconds_target."""
    import oracle
    At = np.ascontiguousarray(A.T)
    threads = oracle.max_threads()
    lg = 22
    while True:
        cnt = 1 << lg
        t0 = time.perf_counter()
        oracle.ryser_range_par(At, 0, cnt - 1, nparts=threads * 4, nthreads=threads)
        dt = time.perf_counter() - t0
        if dt >= seconds_target / 4 or lg >= max_log2:
            if dt < seconds_target and lg < max_log2:
                # one final run sized for the target
                lg2 = min(max_log2, lg + max(0, int(np.log2(seconds_target / max(dt, 1e-3)))))
                if lg2 > lg:
                    lg = lg2
                    cnt = 1 << lg
                    t0 = time.perf_counter()
                    oracle.ryser_range_par(At, 0, cnt - 1, nparts=threads * 4, nthreads=threads)
                    dt = time.perf_counter() - t0
            # one core, for comparison with single-core figures
            t1 = time.perf_counter()
            oracle.ryser_range(At, 0, (1 << 22) - 1)
            single = (1 << 22) / (time.perf_counter() - t1)
            return {"value": cnt / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                    "sample": f"Gray indices 0..2^{lg}-1 of the seeded {A.shape[0]}x{A.shape[0]} matrix "
                              f"({cnt} subsets, {dt:.2f} s wall on {threads} threads)",
                    "single_core_value": single}
        lg += 2


def workload_config() -> dict:
    return {"workload": "perm mod 3 of the seeded uniform 36x36 and 40x40 matrices over F3, "
                        "full 2^n Gray walk, one matrix per launch",
            "sizes": list(SIZES), "subsets_per_step": sum(1 << n for n in SIZES),
            "l2": "flushed between steps (256 MB write); the walk reads < 100 KB per launch"}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    mats = matrices()
    A = mats[36]
    info = cpu_sample(A, seconds_target=6.0)
    per_step = int(info["sample"].split("(")[1].split(" ")[0])
    import oracle
    At = np.ascontiguousarray(A.T)
    th = oracle.max_threads()
    for _ in range(args.warmup):
        oracle.ryser_range_par(At, 0, (1 << 20) - 1, nparts=th * 4, nthreads=th)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ryser_range_par(At, 0, per_step - 1, nparts=th * 4, nthreads=th)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                             "sample": f"each step walks Gray indices 0..{per_step - 1} of the 36x36 matrix "
                                       f"(a bounded sample of the workload; subsets/s is the unit)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2407_20205_gb300 import binding as pf3

    mats = matrices()
    dev = torch.device("cuda", local)
    dA = {n: torch.from_numpy(mats[n]).to(dev) for n in SIZES}
    out = {n: torch.zeros(3, dtype=torch.int64, device=dev) for n in SIZES}
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    from paper_2407_20205_gb300 import multirank
    ranges = {n: multirank.rank_range(n, rank, world) for n in SIZES}

    def step():
        for n in SIZES:
            a, b = ranges[n]
            pf3.perm_f3_range_counts_async(dA[n], n, a, b, out[n], stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    tune = pf3.autotune()  # picks the kernel variants and batch planning (untimed)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()

    # timed region: K steps, each bracketed by events on the launching stream;
    # the L2 flush runs between steps, outside the events
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(SIZES) + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            for j, n in enumerate(SIZES):
                a, b = ranges[n]
                pf3.perm_f3_range_counts_async(dA[n], n, a, b, out[n], stream)
                ev[k][j + 1].record(stream)
    stream.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k][0].elapsed_time(ev[k][-1]) for k in range(args.steps)]
    launch_ms = {n: [ev[k][j].elapsed_time(ev[k][j + 1]) for k in range(args.steps)] for j, n in enumerate(SIZES)}
    total_ms = float(sum(step_ms))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    # results: sum the per-rank counts (the one exchange of the range split)
    counts = {n: out[n][:2].clone() for n in SIZES}
    if world > 1:
        for n in SIZES:
            torch.distributed.all_reduce(counts[n])
    results = {}
    for n in SIZES:
        # the counts are uint64 carried in int64 tensors: read the bits back unsigned
        p, m = [int(x) % (1 << 64) for x in counts[n].cpu()]
        results[n] = pf3.perm_from_counts(n, p, m)
    subsets_step = sum(1 << n for n in SIZES)
    value = subsets_step * args.steps / (total_ms * 1e-3)

    # e2e through the public host-pointer API.  N = 1: perm_f3 per matrix
    # (input copied in, result out, every call).  N > 1: every rank walks its
    # Gray range with perm_f3_range_counts (copies in and out every call), the
    # counts are summed across ranks and the library maps them to the result.
    e2e_dt = None
    if world == 1:
        for n in SIZES:
            pf3.perm_f3(mats[n])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for n in SIZES:
                r = pf3.perm_f3(mats[n])
                assert r == results[n]
        e2e_dt = time.perf_counter() - t0
    else:
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for n in SIZES:
                a, b = ranges[n]
                p, m = pf3.perm_f3_range_counts(mats[n], a, b) if a <= b else (0, 0)
                P, M = multirank.allreduce_counts(p, m, device=dev)
                assert pf3.perm_from_counts(n, P, M) == results[n]
        barrier()
        t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_dt = float(t.item())

    line = None
    if rank == 0:
        pk = peaks()
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        info = pf3.device_info()
        n_sm = info["sm_count"]
        # roofline of the dominant kernel (the W = 2 walk, both launches)
        g_single = pf3.variant_info(pf3.SINGLE, pf3.get_variant(pf3.SINGLE, 2))["G"]
        ops = sum((1 << n) // world * i_alg(g_single) for n in SIZES) * args.steps
        kern_s = sum(sum(v) for v in launch_ms.values()) * 1e-3
        achieved = ops / kern_s / 1e12
        lanes = float(os.environ.get("PF3_ALU_LANES", "64"))
        peak = n_sm * sm_max * 1e6 * lanes / 1e12
        prof = profiled()
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": prof.get("dram_bytes_per_launch"),
                "ops_per_subset": i_alg(g_single),
                "executed_alu_inst_per_subset": prof.get("alu_inst_per_subset"),
                "alu_pipe_busy": prof.get("alu_pipe_busy"),
                "note": f"ops = {i_alg(g_single):.4f} minimal ALU instructions per subset (grouped walk, "
                        f"G = {g_single}; probes of 2 LOP3 + half a predicate OR); peak = {n_sm} SMs x "
                        f"{sm_max:.0f} MHz x {lanes:.0f} lanes/clk/SM (ALU pipe issue), of measured clock; "
                        f"executed ALU instructions per subset and ALU pipe busy are ncu figures of this kernel"}
        # e2e through the host-pointer C entry point (copies in and out each call)
        e2e = {"value": subsets_step * args.steps / e2e_dt, "unit": UNIT,
               "h2d_bytes_per_step": int(world * sum(n * n for n in SIZES)),
               "d2h_bytes_per_step": int(world * 24 * len(SIZES)),
               "path": "perm_f3 per matrix" if world == 1 else
                       "perm_f3_range_counts per rank, counts summed across ranks, pf3_perm_from_counts"}
        extra = {}
        if not args.no_batch and world == 1:
            extra["batch_n24"] = bench_batch(pf3, torch, dev, stream)
            extra["batch_n24"]["one_matrix_per_launch"] = bench_single_launches(pf3, torch, dev, stream)
        if not args.no_serve and world == 1:
            from paper_2407_20205_gb300 import serve
            out, _, _ = serve.run(jobs=args.serve_jobs, nmin=12, nmax=40, rho=0.7, capacity=value)
            extra["serve"] = out
        if world == 1:
            extra["dense_vs_grouped_n39"] = bench_dense(pf3, torch, dev, stream)
        if not args.no_config1 and world == 1:
            extra["config1_n20"] = bench_n20(pf3, torch, dev, stream)
        if not args.no_long and world == 1:
            extra["long_n48"] = bench_long(pf3)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_sample(mats[36])
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {**workload_config(),
                           "results": {str(n): results[n] for n in SIZES},
                           "ms_per_launch": {str(n): float(np.mean(v)) for n, v in launch_ms.items()},
                           "parallelism": f"range split x{world}" if world > 1 else "1 GPU",
                           "variants": {"single": tune["single_variant"],
                                        "single_short_launches": tune["single_short_variant"],
                                        "single_merged_columns": tune["single_merged_variant"],
                                        "batch": tune["batch_variant"]},
                           "batch_tuning": tune["batch_tuning"],
                           "autotune_ms": {"single": tune["single_ms"], "batch": tune["batch_ms"],
                                           "pack_packed_vs_warp": {str(n): v for n, v in tune["pack_ms"].items()},
                                           "split_items_per_warp": {str(g): v for g, v in
                                                                    tune["split_ms"].items()}}},
                "clocks": clk, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": len(SIZES) * args.steps, "wall_s_timed": t_wall, "extra": extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_batch(pf3, torch, dev, stream, count=200000):
    """Batched Monte Carlo: 200,000 seeded uniform 24x24 matrices, one call."""
    from paper_2407_20205_gb300 import inputs
    A = inputs.uniform_matrices(inputs.SEED_BATCH24, 24, count)
    ns = np.full(count, 24, dtype=np.int32)
    dAs = torch.from_numpy(A.reshape(-1)).to(dev)
    dres = torch.zeros(count, dtype=torch.uint8, device=dev)
    dh = torch.zeros(3, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        pf3.perm_f3_batch_async(dAs, ns, dres, dh, stream)  # warm-up
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pf3.perm_f3_batch_async(dAs, ns, dres, dh, stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    hist = [int(x) for x in dh.cpu()]
    sub_s = count * (1 << 24) / (ms * 1e-3)
    n_sm = pf3.device_info()["sm_count"]
    peak_ops = n_sm * float(peaks().get("sm_max_mhz", 2070.0)) * 1e6 * 64
    g_batch = pf3.variant_info(pf3.BATCH, pf3.get_variant(pf3.BATCH, 1))["G"]
    return {"matrices": count, "n": 24, "ms": ms, "perms_per_s": count / (ms * 1e-3),
            "subsets_per_s": sub_s, "hist": hist,
            "alu_frac": sub_s * i_alg(g_batch) / peak_ops, "alu_ops_per_subset": i_alg(g_batch)}


def bench_single_launches(pf3, torch, dev, stream, count=2000):
    """The plain form for comparison: the same n = 24 matrices, one launch each."""
    from paper_2407_20205_gb300 import inputs
    A = inputs.uniform_matrices(inputs.SEED_BATCH24, 24, count)
    dA = torch.from_numpy(A).to(dev)
    out = torch.zeros((count, 3), dtype=torch.int64, device=dev)
    last = (1 << 24) - 1
    with torch.cuda.stream(stream):
        for k in range(8):
            pf3.perm_f3_range_counts_async(dA[k], 24, 0, last, out[k], stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(count):
            pf3.perm_f3_range_counts_async(dA[k], 24, 0, last, out[k], stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    return {"matrices": count, "ms": ms, "perms_per_s": count / (ms * 1e-3),
            "subsets_per_s": count * (1 << 24) / (ms * 1e-3)}


def alu_peak_ops(pf3):
    """ALU-pipe lane-instructions per second of the whole GPU at the measured
    maximum SM clock (64 lanes per clock per SM)."""
    n_sm = pf3.device_info()["sm_count"]
    return n_sm * float(peaks().get("sm_max_mhz", 2070.0)) * 1e6 * 64


def bench_n20(pf3, torch, dev, stream, launches=200):
    """The seeded uniform 20 x 20 matrix: all 2^20 Gray indices, one matrix per
    launch, timed over `launches` back-to-back launches with CUDA events on
    the launching stream (a launch this short is bound by its fixed costs)."""
    from paper_2407_20205_gb300 import inputs
    A = inputs.uniform_matrix(inputs.SEED_N20, 20)
    dA = torch.from_numpy(A).to(dev)
    out = torch.zeros(3, dtype=torch.int64, device=dev)
    last = (1 << 20) - 1
    with torch.cuda.stream(stream):
        for _ in range(5):
            pf3.perm_f3_range_counts_async(dA, 20, 0, last, out, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(launches):
            pf3.perm_f3_range_counts_async(dA, 20, 0, last, out, stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / launches
    g = pf3.variant_info(pf3.SINGLE, pf3.get_variant(pf3.SINGLE_SHORT, 1))["G"]
    sub_s = (1 << 20) / (ms * 1e-3)
    p, m, r = [int(x) % (1 << 64) for x in out.cpu()]
    return {"n": 20, "launches": launches, "ms_per_launch": ms, "subsets_per_s": sub_s, "perms_per_s": 1e3 / ms,
            "perm": r, "alu_frac": sub_s * i_alg(g) / alu_peak_ops(pf3), "alu_ops_per_subset": i_alg(g)}


def bench_dense(pf3, torch, dev, stream, n=39, reps=3):
    """The dense walk against the grouped walk at one size: J_n (all ones, two
    thirds of its terms nonzero, every warp in the dense walk) and the seeded
    uniform n x n matrix, each a full 2^n walk in one launch through the
    device-pointer call (A as it is), and J_n through the host-pointer call,
    which merges its equal columns first and then either walks the merged
    matrix (class limit 0) or counts it by column-sum vector (the default)."""
    from paper_2407_20205_gb300 import inputs
    out = torch.zeros(3, dtype=torch.int64, device=dev)
    res = {}
    for name, A in (("ones", np.ones((n, n), np.uint8)), ("uniform", inputs.uniform_matrix(3900 + n, n))):
        dA = torch.from_numpy(A).to(dev)
        last = (1 << n) - 1
        with torch.cuda.stream(stream):
            pf3.perm_f3_range_counts_async(dA, n, 0, last, out, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                pf3.perm_f3_range_counts_async(dA, n, 0, last, out, stream)
            e1.record(stream)
        stream.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1) / reps, "perm": int(out[2].cpu())}
    # the host-pointer call on J_n: its equal columns merge into one or two,
    # which are counted by column-sum vector; with the class limit at 0 the
    # merged matrix (one plane word) is walked.  Wall clock around perm_f3,
    # copies included.
    J = np.ones((n, n), np.uint8)
    keep = pf3.get_class_limit()
    for key, limit in (("ones_merged_host_call", 0), ("ones_by_class_host_call", keep)):
        pf3.set_class_limit(limit)
        try:
            pf3.perm_f3(J)
            t = []
            for _ in range(reps):
                t0 = time.perf_counter()
                r = pf3.perm_f3(J)
                t.append((time.perf_counter() - t0) * 1e3)
        finally:
            pf3.set_class_limit(keep)
        res[key] = {"ms": float(min(t)), "perm": r}
    res["n"] = n
    res["ratio"] = res["ones"]["ms"] / res["uniform"]["ms"]
    res["ratio_merged"] = res["ones_merged_host_call"]["ms"] / res["uniform"]["ms"]
    res["ratio_by_class"] = res["ones_by_class_host_call"]["ms"] / res["uniform"]["ms"]
    return res


def bench_long(pf3):
    """48 x 48 seeded uniform matrix, all 2^48 Gray indices in bounded launches
    of 2^44 (16 launches, each followed by a host read of its counts)."""
    from paper_2407_20205_gb300 import inputs
    A = inputs.uniform_matrix(inputs.SEED_N48, 48)
    t0 = time.perf_counter()
    r = pf3.longrun(A, chunk_log2=44)
    dt = time.perf_counter() - t0
    g = pf3.variant_info(pf3.SINGLE, pf3.get_variant(pf3.SINGLE, 2))["G"]
    sub_s = (1 << 48) / dt
    return {"n": 48, "seconds": dt, "subsets_per_s": sub_s, "perm": r.get("perm"),
            "plus": r["plus"], "minus": r["minus"], "launches": 1 << 4,
            "alu_frac": sub_s * i_alg(g) / alu_peak_ops(pf3), "alu_ops_per_subset": i_alg(g),
            "timing": "host wall clock around pf3_longrun (includes 16 synchronising count reads)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=5000)
    ap.add_argument("--no-config1", action="store_true", help="skip the seeded 20x20 matrix")
    ap.add_argument("--no-long", action="store_true", help="skip the seeded 48x48 matrix (about 40 s)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

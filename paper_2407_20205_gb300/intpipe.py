"""Integer-pipe issue-rate microbenchmark (roofline denominator of the walk).

    python -m paper_2407_20205_gb300.intpipe [--ctas-per-sm 8] [--threads 256]

Prints one JSON object: for each instruction kind, thread instructions per
clock per SM and the SM clock the CTAs saw, plus the walk step's subsets per
clock per SM (the step is three LOP3 and one compare per 32-bit word).
"""
from __future__ import annotations

import argparse
import json


def run(ctas_per_sm=8, threads=256, iters=4096):
    from . import binding
    res = {"device": binding.device_info()}
    for kind in binding.INTPIPE_KINDS:
        r = binding.intpipe_bench(kind, ctas_per_sm=ctas_per_sm, threads=threads, iters=iters)
        res[kind] = r
    # lanes per clock per SM from the whole-GPU rate and the clock the CTAs saw
    sm = res["device"]["sm_count"]
    for kind in binding.INTPIPE_KINDS:
        r = res[kind]
        r["lanes_per_clk_per_sm_wall"] = r["inst_per_s"] / (sm * r["sm_mhz"] * 1e6) if r["sm_mhz"] else None
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ctas-per-sm", type=int, default=8)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--iters", type=int, default=4096)
    a = ap.parse_args()
    out = {}
    for cps in sorted({2, 4, a.ctas_per_sm}):
        out[f"ctas_per_sm={cps}"] = run(cps, a.threads, a.iters)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()

"""Monte Carlo estimates of P(perm(A) = 0) for uniform random A in F3^{n x n}
(Sec. 4, Table 3), through the batch entry point on the GPU.

    python -m paper_2407_20205_gb300.montecarlo --ns 6,8,10,12,16,20,24,28 --budget 1e12

For each n it draws `trials` seeded uniform matrices (trials = min(max_trials,
budget / 2^n)), runs them as one batch and reports the zero count with the
paper's estimate and the binomial z-score of the difference.
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

from . import binding, inputs

SEED_MC = 3000


def paper_table():
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        "table3_montecarlo.txt")
    rows = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            n, z, lg = line.split()
            rows[int(n)] = int(z) / 10 ** int(lg)
    return rows


def estimate(n: int, trials: int, seed: int = SEED_MC, chunk: int = 200000):
    zeros = ones = twos = 0
    done = 0
    while done < trials:
        cnt = min(chunk, trials - done)
        A = inputs.uniform_matrices(seed + n, n, cnt, start=done)
        res, hist = binding.perm_f3_batch(flat=A.reshape(-1), ns=np.full(cnt, n, np.int32), with_hist=True)
        zeros += int(hist[0])
        ones += int(hist[1])
        twos += int(hist[2])
        done += cnt
    return zeros, ones, twos


def run(ns, budget=1e12, max_trials=10 ** 6):
    table = paper_table()
    out = []
    for n in ns:
        trials = int(max(1000, min(max_trials, budget / (1 << n))))
        z, o, t = estimate(n, trials)
        p_hat = z / trials
        row = {"n": n, "trials": trials, "zeros": z, "ones": o, "twos": t, "p0": p_hat}
        if n in table:
            p = table[n]
            sd = math.sqrt(p * (1 - p) / trials)
            row.update({"paper_p0": p, "z_vs_paper": (p_hat - p) / sd,
                        "z_vs_third": (p_hat - 1 / 3) / math.sqrt((1 / 3) * (2 / 3) / trials)})
        out.append(row)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ns", default="6,7,8,10,12,16,20,24,28")
    ap.add_argument("--budget", type=float, default=1e12)
    ap.add_argument("--max-trials", type=int, default=10 ** 6)
    a = ap.parse_args()
    print(json.dumps(run([int(x) for x in a.ns.split(",")], a.budget, a.max_trials)))


if __name__ == "__main__":
    main()

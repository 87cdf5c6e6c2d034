"""One small, self-contained launch for profilers.

    python -m paper_2407_20205_gb300.profile_case --kind single --n 36
    python -m paper_2407_20205_gb300.profile_case --kind batch --n 24 --count 2000
    python -m paper_2407_20205_gb300.profile_case --kind ones --n 40
    python -m paper_2407_20205_gb300.profile_case --kind classes --n 40

single: perm of the seeded uniform n x n matrix (one launch of the walk);
batch: one batch call over `count` seeded uniform n x n matrices;
ones: perm of the all-ones matrix J_n, walked (one launch; two thirds of its
terms are nonzero, so every warp walks it with the dense walk; for n > 32 its
columns merge into one or two, walked on one plane word: the class limit is
set to 0 so that the matrix is not counted by column-sum vector);
classes: perm of an n x n matrix (n > 32) with columns drawn from two pools
of two vectors each, whose columns merge into at most 8: one launch of the
count by column-sum vector.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="single", choices=["single", "batch", "ones", "classes"])
    ap.add_argument("--n", type=int, default=36)
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=None)
    a = ap.parse_args()
    from . import binding, inputs
    if a.kind == "single":
        seed = a.seed if a.seed is not None else a.n
        r = binding.perm_f3(inputs.uniform_matrix(seed, a.n))
        print(f"perm mod 3 = {r}")
    elif a.kind == "ones":
        binding.set_class_limit(0)
        r = binding.perm_f3(np.ones((a.n, a.n), np.uint8))
        print(f"perm mod 3 = {r}")
    elif a.kind == "classes":
        seed = a.seed if a.seed is not None else 9000 + a.n
        A = inputs.pooled_columns(seed, a.n, 2, 2)
        merged = binding.column_merge(A)
        if merged is None or merged[0].shape[1] > binding.get_class_limit():
            raise SystemExit("the columns do not merge into a narrow matrix: pick another seed")
        r = binding.perm_f3(A)
        print(f"merged columns = {merged[0].shape[1]}, perm mod 3 = {r}")
    else:
        seed = a.seed if a.seed is not None else inputs.SEED_BATCH24
        A = inputs.uniform_matrices(seed, a.n, a.count)
        res, hist = binding.perm_f3_batch(flat=A.reshape(-1), ns=np.full(a.count, a.n, np.int32),
                                          with_hist=True)
        print(f"hist = {list(hist)}")


if __name__ == "__main__":
    main()

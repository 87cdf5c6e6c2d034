"""Command line for the library.

    python -m paper_2407_20205_gb300 perm FILE        # FILE or "-": one row per line,
                                                     # entries in {-1,0,1} or {0,1,2}
    python -m paper_2407_20205_gb300 counts FILE      # also the +1 / -1 Ryser term counts
    python -m paper_2407_20205_gb300 random N SEED    # a seeded uniform N x N matrix
    python -m paper_2407_20205_gb300 table2 N         # counts of perm = 0, 1, 2 over F3^{N x N}
    python -m paper_2407_20205_gb300 autotune

Results are perm(A) mod 3 in {0, 1, 2} (2 stands for -1).
"""
from __future__ import annotations

import json
import sys

import numpy as np


def read_matrix(path: str) -> np.ndarray:
    text = sys.stdin.read() if path == "-" else open(path).read()
    rows = [[int(x) for x in line.split()] for line in text.splitlines() if line.strip()]
    A = np.array(rows, dtype=np.int64)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise SystemExit("a square matrix is expected (one row per line)")
    if A.min() < -1 or A.max() > 2:
        raise SystemExit("entries must be in {-1, 0, 1} or {0, 1, 2}")
    return (A % 3).astype(np.uint8)


def main(argv=None):
    argv = list(sys.argv[1:] if argv is None else argv)
    if not argv or argv[0] in ("-h", "--help"):
        print(__doc__)
        return 0
    from . import binding, inputs
    cmd = argv[0]
    if cmd == "perm":
        print(binding.perm_f3(read_matrix(argv[1] if len(argv) > 1 else "-")))
    elif cmd == "counts":
        A = read_matrix(argv[1] if len(argv) > 1 else "-")
        p, m = binding.perm_f3_counts(A)
        print(json.dumps({"n": int(A.shape[0]), "plus": p, "minus": m,
                          "perm": binding.perm_from_counts(int(A.shape[0]), p, m)}))
    elif cmd == "random":
        n, seed = int(argv[1]), int(argv[2])
        for row in inputs.uniform_matrix(seed, n):
            print(" ".join(str(int(v)) for v in row))
    elif cmd == "table2":
        c = binding.count_exhaustive(int(argv[1]))
        print(json.dumps({"n": int(argv[1]), "perm0": c[0], "perm1": c[1], "perm2": c[2]}))
    elif cmd == "autotune":
        print(json.dumps(binding.autotune()))
    else:
        raise SystemExit(f"unknown command {cmd!r}; see --help")
    return 0


if __name__ == "__main__":
    sys.exit(main())

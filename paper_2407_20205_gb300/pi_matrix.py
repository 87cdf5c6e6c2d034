"""The digit matrix Pi_n of Sec. 3.1 and its permanent mod 3.

Sec. 3.1 reports perm(Pi_50) = -1 (mod 3), where the (i, j) entry of Pi_n is a
decimal digit of pi and "the first row are the first n digits of pi".  That
fixes entry (i, j) (1-based) as digit number n(i - 1) + j, counting the
leading 3 as digit 1 ("with_three"); the other reading starts at the first
digit after the decimal point ("after_point").  A digit d is the F3 element
d mod 3.

Digits are computed here with integer arithmetic: Machin's formula
pi = 16 arctan(1/5) - 4 arctan(1/239), arctan(1/x) by its alternating series,
with guard digits.

    python -m paper_2407_20205_gb300.pi_matrix --n 50 --reading with_three \
        --checkpoint pi50.ckpt
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def _arctan_inv(x: int, unity: int) -> int:
    """unity * arctan(1/x) by the alternating series."""
    total = term = unity // x
    x2 = x * x
    k = 1
    sign = -1
    while term:
        term //= x2
        total += sign * (term // (2 * k + 1))
        sign = -sign
        k += 1
    return total


def pi_digits_machin(count: int) -> str:
    """The first `count` decimal digits of pi ("314159...")."""
    guard = 20
    unity = 10 ** (count + guard)
    pi = 4 * (4 * _arctan_inv(5, unity) - _arctan_inv(239, unity))
    return str(pi)[:count]


def digit_matrix(n: int, reading: str = "with_three") -> np.ndarray:
    start = 0 if reading == "with_three" else 1
    digits = pi_digits_machin(n * n + start + 5)
    d = np.frombuffer(digits[start:start + n * n].encode(), dtype=np.uint8) - ord("0")
    return (d.reshape(n, n) % 3).astype(np.uint8)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=50)
    ap.add_argument("--reading", default="with_three", choices=["with_three", "after_point"])
    ap.add_argument("--chunk-log2", type=int, default=44)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--max-seconds", type=float, default=0.0)
    a = ap.parse_args()
    from . import binding
    A = digit_matrix(a.n, a.reading)
    t0 = time.perf_counter()
    r = binding.longrun(A, chunk_log2=a.chunk_log2, checkpoint=a.checkpoint, max_seconds=a.max_seconds)
    r["seconds"] = time.perf_counter() - t0
    r.update({"n": a.n, "reading": a.reading})
    if r["finished"]:
        r["subsets_per_s"] = (1 << a.n) / r["seconds"]
    print(json.dumps(r))


if __name__ == "__main__":
    main()

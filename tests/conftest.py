import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def oracle():
    import oracle as _o
    _o.lib()
    return _o


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden(name):
    """Rows of whitespace-separated fields; '#' lines are comments/citations."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def rank_one_counts(d, e):
    """Exact (plus, minus) of the row-subset Ryser terms of A_ij = d_i e_j
    (d, e in {1, -1}): the row sums over S are e_j t with t = sum_{i in S} d_i,
    so the term of S is (-1)^|S| (prod e) t^n, nonzero iff t != 0 mod 3.
    Counted by the split (a, b) of S over the rows with d = +1 and d = -1."""
    n = len(e)
    p = sum(1 for x in d if x == 1)
    q = len(d) - p
    pe = 1
    for x in e:
        pe *= x
    plus = minus = 0
    for a in range(p + 1):
        for b in range(q + 1):
            t = (a - b) % 3
            if t == 0:
                continue
            tt = 1 if t == 1 else -1
            sign = (-1) ** (a + b) * pe * tt ** n
            cnt = math.comb(p, a) * math.comb(q, b)
            if sign > 0:
                plus += cnt
            else:
                minus += cnt
    return plus, minus

"""The column merge of the host-pointer single-matrix calls, on the CPU (a
host function of the library; no device): columns equal up to a factor -1
become one class, kept once (odd multiplicity) or twice (even), and every
Ryser term of the merged n x m matrix is A's times (-1)^negate.  Checked
against the oracle: plain per-index terms of the merged matrix, summed over
Gray windows, equal the oracle's counts of A (swapped when negate)."""
import numpy as np
import pytest

from paper_2407_20205_gb300 import inputs


@pytest.fixture(scope="module")
def pf3():
    from paper_2407_20205_gb300 import build
    build.build()
    from paper_2407_20205_gb300 import binding
    return binding


def window_counts(X, first, last):
    """(plus, minus) of the row-subset Ryser terms of the n-row matrix X over
    Gray indices first..last, by direct evaluation of each subset sum."""
    n = X.shape[0]
    i = np.arange(first, last + 1, dtype=np.uint64)
    g = i ^ (i >> np.uint64(1))
    rows = ((g[:, None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
    sums = (rows @ X.astype(np.int64)) % 3
    vals = np.where(sums == 2, -1, sums)
    prod = vals.prod(axis=1) * np.where(rows.sum(axis=1) % 2 == 1, -1, 1)
    return int((prod == 1).sum()), int((prod == -1).sum())


def test_ones_and_rank_one(pf3):
    for n in (33, 34, 40, 63, 64):
        B, neg = pf3.column_merge(np.ones((n, n), np.uint8))
        assert B.shape == (n, 1 if n % 2 else 2) and not neg and (B == 1).all()
    rng = np.random.default_rng(5)
    for n in (35, 48):
        d, e = rng.choice([1, 2], n), rng.choice([1, 2], n)
        A = (np.outer(d, e) % 3).astype(np.uint8)
        B, neg = pf3.column_merge(A)
        assert B.shape[1] in (1, 2)
        assert neg == bool(((e * d[0]) % 3 == 2).sum() % 2)


def test_no_merge_when_it_does_not_pay(pf3):
    assert pf3.column_merge(inputs.uniform_matrix(3, 40)) is None      # all columns distinct
    assert pf3.column_merge(np.ones((20, 20), np.uint8)) is None       # one word already
    A = inputs.pooled_columns(11, 64, 30, None)                        # more than 32 columns left
    assert pf3.column_merge(A) is None


@pytest.mark.parametrize("n,pool", [(33, 2), (36, 3), (40, 4), (45, 5), (64, 5)])
def test_merged_terms_match_the_oracle(pf3, oracle, n, pool):
    A = inputs.pooled_columns(8800 + n, n, pool, pool)
    merged = pf3.column_merge(A)
    assert merged is not None
    B, neg = merged
    assert B.shape[0] == n and B.shape[1] <= 32
    rng = np.random.default_rng(n)
    nonzero = 0
    for first in (0, int(rng.integers(0, 1 << 30)) * 7 + 3):
        last = first + 6000
        want = oracle.ryser_range(np.ascontiguousarray(A.T), first, last)
        got = window_counts(B, first, last)
        assert ((got[1], got[0]) if neg else got) == want
        nonzero += sum(want)
    assert nonzero > 100


def test_class_counts_refusals_touch_no_device(pf3):
    """pf3_class_counts merges on the host first: a matrix whose columns merge
    into more than 8 is left to the walk (None) and a bad entry or size is an
    error, all before any device is needed."""
    assert pf3.class_counts(inputs.uniform_matrix(inputs.SEED_N20, 20)) is None
    # 9 distinct columns (no two equal up to sign), n = 9
    A = np.zeros((9, 9), np.uint8)
    for j in range(9):
        A[j, j] = 1
    assert pf3.class_counts(A) is None
    bad = np.ones((5, 5), np.uint8)
    bad[1, 1] = 7
    with pytest.raises(pf3.PF3Error) as ei:
        pf3.class_counts(bad)
    assert ei.value.code == pf3.PF3_EDOMAIN
    assert pf3._lib_class_counts(None, 4, None, None) == pf3.PF3_EINVAL
    with pytest.raises(pf3.PF3Error):
        pf3.class_counts(np.zeros((65, 65), np.uint8))

"""Ryser counts by column-sum vector (pf3_class_counts, and the routes that
take it: perm_f3 / perm_f3_counts for n > 32, a fresh long run, serving)
against the oracle, closed forms, and the Gray walk over the same matrix.

A term of Eq. (2) depends on its row subset only through the column sums and
the parity of the subset's size; the device counts the subsets on each of
those pairs row by row.  The counts must be exactly the walk's."""
import os

import numpy as np
import pytest

from paper_2407_20205_gb300 import inputs

from conftest import rank_one_counts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    return binding


def _full(n):
    return (1 << n) - 1


def _pooled(seed, n, pool):
    """n x n (n <= 32) with every column a random multiple (1 or 2) of one of
    `pool` random vectors: at most `pool` column classes."""
    return inputs.pooled_columns(seed, n, pool, None)


def test_small_matrices_vs_oracle(pf3, oracle):
    """Every matrix of n <= 8 has at most 8 merged columns: counted on the
    device, compared count for count with the oracle (A^T: the oracle sums
    over column subsets) -- uniform entries, zero rows and zero columns."""
    rng = np.random.default_rng(8100)
    for trial in range(120):
        n = 1 + trial % 8
        A = rng.integers(0, 3, size=(n, n)).astype(np.uint8)
        if trial % 3 == 0:
            A[:, rng.integers(0, n)] = 0
        if trial % 5 == 0:
            A[rng.integers(0, n), :] = 0
        got = pf3.class_counts(A)
        assert got is not None
        assert got == oracle.ryser_range(np.ascontiguousarray(A.T), 0, _full(n)), (trial, n)


@pytest.mark.parametrize("n", [9, 12, 16, 20, 24])
def test_pooled_columns_vs_oracle(pf3, oracle, n):
    """Few column classes at n up to 24 (2^24 oracle terms), with random
    signs per column (the merge's sign swap): counts equal the oracle's."""
    for pool in (1, 2, 3, 4):
        A = _pooled(8200 + 10 * n + pool, n, pool)
        got = pf3.class_counts(A)
        assert got is not None, (n, pool)
        want = oracle.ryser_range_par(np.ascontiguousarray(A.T), 0, _full(n))
        assert got == want, (n, pool)


def test_wide_matrix_is_not_counted(pf3):
    """A matrix whose columns merge into more than 8 is left to the walk."""
    A = inputs.uniform_matrix(inputs.SEED_N20, 20)
    assert pf3.class_counts(A) is None
    bad = np.ones((5, 5), np.uint8)
    bad[2, 3] = 3
    with pytest.raises(pf3.PF3Error):
        pf3.class_counts(bad)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 20, 33, 39, 40, 47, 63, 64])
def test_rank_one_closed_form_by_class(pf3, n):
    """J_n and D1 J D2 (random signs): one or two merged columns; the counts
    have a closed form (the column sums over S are e_j times a signed count
    of S), also at n = 64 where they approach 2^63 -- through
    pf3_class_counts and, for n > 32, through perm_f3_counts and perm_f3."""
    rng = np.random.default_rng(8300 + n)
    J = np.ones((n, n), np.uint8)
    d = rng.choice([1, -1], size=n)
    e = rng.choice([1, -1], size=n)
    D = (np.outer(d, e) % 3).astype(np.uint8)
    for A, want in ((J, rank_one_counts([1] * n, [1] * n)), (D, rank_one_counts(list(d), list(e)))):
        assert pf3.class_counts(A) == want
        if n > 32:
            assert pf3.perm_f3_counts(A) == want
            assert pf3.perm_f3(A) == ((want[0] - want[1]) * (-1) ** n) % 3


@pytest.mark.parametrize("n", [33, 34, 35, 36])
def test_route_equals_walk(pf3, n):
    """For n > 32 the host-pointer calls count narrow merged matrices by
    column-sum vector; with the class limit at 0 they walk the same merged
    matrix: both give the same counts (pooled columns with random signs, two
    pools of 2 vectors, so at most 4 classes and a merged width of at most 8)."""
    A = inputs.pooled_columns(8400 + n, n, 2, 2)
    merged = pf3.column_merge(A)
    assert merged is not None and merged[0].shape[1] <= 8
    routed = pf3.perm_f3_counts(A)
    keep = pf3.get_class_limit()
    try:
        pf3.set_class_limit(0)
        walked = pf3.perm_f3_counts(A)
    finally:
        pf3.set_class_limit(keep)
    assert routed == walked
    assert pf3.class_counts(A) == walked


def test_limit_api(pf3):
    keep = pf3.get_class_limit()
    assert keep == pf3.CLASS_MAX_COLS
    for bad in (-1, pf3.CLASS_MAX_COLS + 1):
        with pytest.raises(pf3.PF3Error):
            pf3.set_class_limit(bad)
    assert pf3.get_class_limit() == keep


def test_longrun_by_class(pf3, tmp_path):
    """A fresh long run of J_45 finishes in one call by column-sum vector,
    with the closed-form counts and a finished checkpoint.  A run stopped
    part-way (walked, class limit 0) resumes from its checkpoint with the
    walk and ends with the same closed-form counts."""
    n = 45
    J = np.ones((n, n), np.uint8)
    want = rank_one_counts([1] * n, [1] * n)
    ck = str(tmp_path / "j45.ck")
    r = pf3.longrun(J, chunk_log2=30, checkpoint=ck)
    assert r["finished"] and (r["plus"], r["minus"]) == want
    assert r["perm"] == ((want[0] - want[1]) * (-1) ** n) % 3
    assert "done=1" in open(ck).read()
    n = 36
    J = np.ones((n, n), np.uint8)
    want = rank_one_counts([1] * n, [1] * n)
    ck2 = str(tmp_path / "j36.ck")
    keep = pf3.get_class_limit()
    try:
        pf3.set_class_limit(0)
        r = pf3.longrun(J, chunk_log2=34, checkpoint=ck2, max_seconds=1e-9)
    finally:
        pf3.set_class_limit(keep)
    assert not r["finished"] and r["next_index"] == 1 << 34
    r = pf3.longrun(J, chunk_log2=34, checkpoint=ck2)
    assert r["finished"] and (r["plus"], r["minus"]) == want
    os.remove(ck2)


def test_serving_by_class(pf3):
    """Serving counts requests whose merged matrix is narrow in the launch
    that admits them: results equal perm_f3's and the closed forms, mixed
    with walked requests, and equal the walked results with the class route
    off (class_max_cols = 0)."""
    rng = np.random.default_rng(8500)
    mats, want = [], []
    for k in range(24):
        n = 33 + k % 8
        if k % 3 == 0:
            d = rng.choice([1, -1], size=n)
            e = rng.choice([1, -1], size=n)
            A = (np.outer(d, e) % 3).astype(np.uint8)
            p, m = rank_one_counts(list(d), list(e))
            want.append(((p - m) * (-1) ** n) % 3)
        elif k % 3 == 1:
            A = inputs.pooled_columns(8600 + k, n, 2, 2)
            want.append(pf3.perm_f3(A))
        else:
            A = inputs.uniform_matrix(8700 + k, 20 + k % 6)
            want.append(pf3.perm_f3(A))
        mats.append(A)
    for limit in (pf3.CLASS_MAX_COLS, 0):
        with pf3.ServeContext(class_max_cols=limit, chunk_log2=24, launch_budget=1 << 32) as ctx:
            tickets = [ctx.submit(A) for A in mats]
            got = [ctx.wait(t) for t in tickets]
        assert got == want, limit

"""Two-word (33 <= n <= 64) parity on inputs whose windows hold nonzero terms.

For a uniform n x n matrix a Ryser term is nonzero with probability about
(2/3)^n, so short windows at n >= 33 hold almost no nonzero terms and a
comparison there only checks zeros.  The tests here compare the CUDA path's
exact (+1, -1) counts with the oracle's on windows that contain many nonzero
terms, and assert that they do:

* 2^30-index windows of the seeded 36 x 36 and 40 x 40 benchmark matrices
  (about 490 and 97 nonzero terms expected), and the whole 2^36 / 2^40 walk
  in the launch configuration the benchmark times, checked as the sum of
  its 2^30 / 2^34 windows;
* engineered matrices at n = 40 and n = 64 whose first 32 columns repeat a
  few column vectors, so that many states pass the first-word zero test
  (Sec. 3: a term is nonzero only when every mag bit is 1) and the second
  word both passes and fails.  One mix keeps the share of probe groups that
  pass below the dense-walk switch (queued exact replay of marked groups),
  one far above it (dense walk); the share is measured here on a sample.

Integer work: tolerance 0.  The kernels walk row subsets, the oracle the
column subsets of Eq. (2), so the oracle gets A^T.
"""
import numpy as np
import pytest

from paper_2407_20205_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    return binding


def T(A):
    return np.ascontiguousarray(np.asarray(A).T)


def first_word_pass_share(A, G, groups=3000, seed=0):
    """Share of probe groups (2^G consecutive Gray indices) with at least one
    state whose first min(n, 32) column sums are all nonzero, over a random
    sample of groups: the groups the grouped walk marks for exact replay.
    Plain integer sums, independent of both implementations."""
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    hi = (1 << (n - G)) if n < 64 else (1 << 62)
    ks = rng.integers(0, hi, size=groups, dtype=np.uint64)
    j = np.arange(1 << G, dtype=np.uint64)
    idx = (ks[:, None] << np.uint64(G)) | j[None, :]
    gray = idx ^ (idx >> np.uint64(1))
    rows = ((gray[..., None] >> np.arange(n, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
    sums = np.einsum("gjr,rc->gjc", rows, A[:, :32].astype(np.int64)) % 3
    return float((sums != 0).all(axis=2).any(axis=1).mean())


def device_range_counts(pf3, A, a, b):
    """perm_f3_range_counts_async: the device-pointer path, which walks A as
    it is (the host-pointer calls may first merge equal columns)."""
    import torch
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    pf3.perm_f3_range_counts_async(dA, n, a, b, out, None)
    torch.cuda.synchronize()
    return tuple(int(x) % (1 << 64) for x in out[:2].cpu())


def _check_window(pf3, oracle, A, a, b, at_least):
    want = oracle.ryser_range_par(T(A), a, b)
    assert sum(want) >= at_least, (a, b, want)  # the window really holds nonzero terms
    assert pf3.perm_f3_range_counts(A, a, b) == want, (a, b)
    assert device_range_counts(pf3, A, a, b) == want, (a, b)


# ------------------------------------------------------------ the benchmark matrices

@pytest.mark.parametrize("n", [36, 40])
def test_benchmark_matrix_2_30_windows(pf3, oracle, n):
    """Two ragged 2^30-index windows of the seeded benchmark matrix, count for
    count against the oracle, each with at least 25 nonzero terms (50 over
    the pair; about 490 and 97 are expected per window)."""
    seed = inputs.SEED_N36 if n == 36 else inputs.SEED_N40
    A = inputs.uniform_matrix(seed, n)
    rng = np.random.default_rng(900 + n)
    total = 0
    for _ in range(2):
        a = int(rng.integers(0, (1 << n) - (1 << 31))) | 1  # odd start: a ragged head
        b = a + (1 << 30) + int(rng.integers(1, 511))        # and a ragged tail
        want = oracle.ryser_range_par(T(A), a, b)
        got = pf3.perm_f3_range_counts(A, a, b)
        assert got == want, (a, b)
        total += sum(want)
    assert total >= 50, total


@pytest.mark.parametrize("n,window_log2", [(36, 30), (40, 34)])
def test_benchmark_matrix_full_walk_is_the_sum_of_windows(pf3, oracle, n, window_log2):
    """The whole 2^n walk, in the launch configuration the benchmark times
    (guided chunks from an atomic cursor over a full grid), equals the sum
    of its 2^(n - window_log2) consecutive windows (each walked with fixed
    per-thread shares), and the first window's sub-range [0, 2^30) is the
    oracle's count for count."""
    seed = inputs.SEED_N36 if n == 36 else inputs.SEED_N40
    A = inputs.uniform_matrix(seed, n)
    whole = pf3.perm_f3_counts(A)
    w = 1 << window_log2
    parts = [pf3.perm_f3_range_counts(A, k * w, (k + 1) * w - 1) for k in range(1 << (n - window_log2))]
    assert (sum(p for p, _ in parts), sum(m for _, m in parts)) == whole
    _check_window(pf3, oracle, A, 0, (1 << 30) - 1, 20)


# ------------------------------------------------------------ engineered matrices

ENGINEERED = [
    # (n, low_pool, high_pool, regime)
    (40, 16, None, "replay"),
    (40, 2, None, "dense"),
    (64, 18, 4, "replay"),
    (64, 16, 4, "mixed"),
    (64, 2, 4, "dense"),
]


@pytest.mark.parametrize("n,low_pool,high_pool,regime", ENGINEERED)
def test_engineered_two_word_windows(pf3, oracle, n, low_pool, high_pool, regime):
    """Windows of 2^22 to 2^26 Gray indices with ragged ends, count for count.
    The regimes hold for kernel variant 0 (probe groups of 2^5 indices,
    blocks of 2^9: a warp leaves the grouped walk for the dense walk when a
    block marks at least 129 of its 32 x 16 groups, i.e. about 25 %), which
    the test pins while it walks: in the "replay" mix about a tenth of the
    probe groups pass the first-word test (marked groups are queued and
    replayed exactly, and queues that overflow replay in place); in the
    "dense" mix nearly all do (the warps switch to the dense walk); the
    "mixed" one sits near the switch, so some blocks of a warp's share switch
    and others do not.  In all, the second word fails for most of the states
    that pass the first.  The regimes are those of the device-pointer path,
    which walks A as it is; every window is also walked with the variant the
    autotuner chose, and through the host-pointer call, which may merge equal
    columns first."""
    A = inputs.pooled_columns(6400 + 10 * n + low_pool, n, low_pool, high_pool)
    info = pf3.variant_info(pf3.SINGLE, 0)
    assert (info["U"], info["G"]) == (9, 5)
    share = first_word_pass_share(A, info["G"])
    if regime == "replay":
        assert 0.02 < share < 0.15, share
    elif regime == "mixed":
        assert 0.17 < share < 0.3, share
    else:
        assert share > 0.9, share
    rng = np.random.default_rng(6500 + n + low_pool)
    top = (1 << n) - 1
    windows = []
    for lg in (22, 24, 26):
        a = int(rng.integers(0, 1 << min(n - 2, 62))) * 3 + 1  # not block aligned
        windows.append((a, min(top, a + (1 << lg) + int(rng.integers(1, 1000))), 50))
    # a window that starts at index 0 (the empty set, a head walked one by one)
    windows.append((0, (1 << 22) + 4321, 20))
    if n == 64:
        # and one that ends at the last index, 2^64 - 1
        windows.append((top - (1 << 23) - 77, top, 20))
    tuned = {c: pf3.get_variant(c, 2) for c in (pf3.SINGLE, pf3.SINGLE_SHORT)}
    for a, b, at_least in windows:
        want = oracle.ryser_range_par(T(A), a, b)
        assert sum(want) >= at_least, (a, b, want)  # the window really holds nonzero terms
        try:
            pf3.set_variant(pf3.SINGLE, 2, 0)  # both size classes
            got0 = device_range_counts(pf3, A, a, b)
        finally:
            pf3.set_variant(pf3.SINGLE, 2, tuned[pf3.SINGLE])
            pf3.set_variant(pf3.SINGLE_SHORT, 2, tuned[pf3.SINGLE_SHORT])
        assert got0 == want, (a, b, "variant 0, A as it is")
        assert device_range_counts(pf3, A, a, b) == want, (a, b, "tuned variant, A as it is")
        # the host-pointer call (equal columns merged when that fits one plane word)
        assert pf3.perm_f3_range_counts(A, a, b) == want, (a, b, "host-pointer call")

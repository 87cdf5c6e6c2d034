"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so every comparison is exact (tolerance 0): results in {0,1,2}
and the (+1, -1) Ryser term counts.  The kernels walk ROW subsets (the
paper's code, Sec. 3) while the oracle walks the COLUMN subsets of Eq. (2),
so term counts are compared between A on the GPU and A^T in the oracle.
"""
import math

import numpy as np
import pytest

from conftest import rank_one_counts, read_golden
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


# ------------------------------------------------------------ the row step

def test_step_table_exhaustive(pf3):
    """Every (state, constant, direction): psi(out) = psi(state) +- c (Thm 2.1)."""
    tab = pf3.step_table()

    def psi(m, s):
        return 0 if m == 0 else (1 if s == 0 else 2)

    for state in range(4):
        m, s = state >> 1, state & 1
        for c in range(3):
            for d in range(2):
                mo, so = tab[state, c, d]
                want = (psi(m, s) + (c if d == 0 else -c)) % 3
                assert psi(mo, so) == want, (state, c, d)
                if c == 0 and m == 1:
                    assert (mo, so) == (m, s)  # padding columns stay (1, 0)


def test_step_table_matches_table1(pf3):
    """Table 1: the determined outputs of addition are reproduced exactly; the
    rows printed in red (sum 0) may use either zero representation."""
    tab = pf3.step_table()
    for row in read_golden("table1_addition.txt"):
        a, b, m1, s1, m2, s2, mp, sp, free = map(int, row)
        c = 0 if m2 == 0 else (1 if s2 == 0 else 2)
        if m2 == 0 and s2 == 1:
            continue  # the row constant is never the (0,1) zero (rows come from phi)
        mo, so = tab[(m1 << 1) | s1, c, 0]
        assert mo == mp
        if not free:
            assert so == sp


def test_pack_worked_example(pf3):
    row = read_golden("worked_example.txt")[0]
    entries = [int(x) for x in row[0].split(",")]
    n = len(entries)
    mag_msb, sgn_msb = int(row[1], 16), int(row[2], 16)

    def rev(x):
        return int(format(x, f"0{n}b")[::-1], 2)

    A = np.zeros((n, n), np.uint8)
    A[0] = entries
    mag, sgn = pf3.pack(A)
    assert int(mag[0]) == rev(mag_msb) == 0xB
    assert int(sgn[0]) == rev(sgn_msb) == 0x8


# ------------------------------------------------------------ single matrix

@pytest.mark.parametrize("n", list(range(1, 9)))
def test_small_n_vs_bruteforce(pf3, oracle, n):
    for A in inputs.uniform_matrices(1000 + n, n, 40):
        assert pf3.perm_f3(A) == oracle.perm_bruteforce(A)


@pytest.mark.parametrize("n", list(range(1, 25)))
def test_counts_vs_oracle(pf3, oracle, n):
    count = 6 if n <= 16 else (3 if n <= 21 else 1)
    for A in inputs.uniform_matrices(2000 + n, n, count):
        assert pf3.perm_f3_counts(A) == oracle.counts(T(A))
        assert pf3.perm_f3(A) == oracle.perm_mod3(A)


def test_config_n20_full(pf3, oracle):
    A = inputs.uniform_matrix(inputs.SEED_N20, 20)
    assert pf3.perm_f3_counts(A) == oracle.counts(T(A))
    assert pf3.perm_f3(A) == oracle.perm_mod3(A)


def _ranges(rng, n, k, maxlen):
    top = (1 << n) - 1
    out = [(0, min(top, 300)), (max(0, top - 300), top), (127, 129), (128, 255), (5, 5)]
    for _ in range(k):
        a = int(rng.integers(0, top + 1)) if n < 63 else int(rng.integers(0, 1 << 62)) << 2
        a = min(a, top)
        ln = int(rng.integers(0, maxlen))
        out.append((a, min(top, a + ln)))
    return [(a, b) for a, b in out if a <= b <= top]


@pytest.mark.parametrize("n", [9, 14, 20, 31, 32, 33, 36, 40, 48, 63, 64])
def test_range_counts_vs_oracle(pf3, oracle, n):
    rng = np.random.default_rng(n)
    A = inputs.uniform_matrix(3000 + n, n)
    At = T(A)
    for a, b in _ranges(rng, n, 12, 200000):
        assert pf3.perm_f3_range_counts(A, a, b) == oracle.ryser_range(At, a, b), (a, b)


def test_range_partition_adds_up(pf3):
    """Sec. 3.1: disjoint blocks of Gray states add up to the whole sum."""
    rng = np.random.default_rng(5)
    for n in (18, 27, 34):
        A = inputs.uniform_matrix(4000 + n, n)
        whole = pf3.perm_f3_counts(A)
        top = (1 << n) - 1
        cuts = sorted(set(int(x) for x in rng.integers(1, top, 9)))
        bounds = [0] + cuts + [top + 1]
        tot = [0, 0]
        for a, b in zip(bounds[:-1], bounds[1:]):
            p, m = pf3.perm_f3_range_counts(A, a, b - 1)
            tot[0] += p
            tot[1] += m
        assert tuple(tot) == whole


def test_guided_chunks_match_fixed_shares(pf3):
    """A launch of at least 512 Gray blocks per lane hands its blocks out in
    guided chunks from an atomic cursor; shorter ones give each thread a
    fixed share.  A range just above that size (ragged ends included) must
    count the same as its pieces below it, walked with fixed shares, and
    the whole-matrix walk of a 36 x 36 matrix (guided) must equal the sum of
    its eight 2^33 eighths (fixed shares)."""
    info = pf3.device_info()
    ctas = 2 * info["sm_count"]  # the default W = 2 variant: 2 CTAs of 256 threads per SM
    per_lane = 512 * 512  # blocks of 2^9 indices
    threshold = ctas * 256 * per_lane
    A = inputs.uniform_matrix(4100, 40)
    a = 98765
    b = a + threshold + 3 * (1 << 20) + 777
    whole = pf3.perm_f3_range_counts(A, a, b)
    cuts = [a, a + threshold // 3, a + 2 * (threshold // 3), b + 1]
    tot = [0, 0]
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        p, m = pf3.perm_f3_range_counts(A, lo, hi - 1)
        tot[0] += p
        tot[1] += m
    assert tuple(tot) == whole
    B = inputs.uniform_matrix(4101, 36)
    eighth = 1 << 33
    parts = [pf3.perm_f3_range_counts(B, k * eighth, (k + 1) * eighth - 1) for k in range(8)]
    assert (sum(p for p, _ in parts), sum(m for _, m in parts)) == pf3.perm_f3_counts(B)


def _rank_one(seed, n):
    rng = np.random.default_rng(seed)
    d = rng.choice([1, -1], size=n)
    e = rng.choice([1, -1], size=n)
    A = np.outer(d, e) % 3
    return A.astype(np.uint8), d, e


def _device_counts(pf3, A):
    """Counts over all 2^n indices through the device-pointer path, which
    walks A as it is (the host-pointer calls may merge equal columns)."""
    import torch
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    pf3.perm_f3_range_counts_async(dA, n, 0, (1 << n) - 1, out, None)
    torch.cuda.synchronize()
    return tuple(int(x) % (1 << 64) for x in out[:2].cpu())


@pytest.mark.parametrize("n", [14, 20, 27, 33, 36, 40])
def test_dense_terms_closed_form(pf3, n):
    """Matrices with 2/3 of their terms nonzero (all columns proportional)
    send every warp into the dense walk: the exact counts must equal the
    closed form, for J_n and for D1 J D2 with random signs -- through the
    device-pointer path (A as it is: two plane words for n > 32) and the
    host-pointer one (for n > 32 the columns merge into one or two, which are
    counted by column-sum vector; with the class limit at 0 the merged matrix
    is walked)."""
    J = np.ones((n, n), np.uint8)
    A, d, e = _rank_one(7000 + n, n)
    keep = pf3.get_class_limit()
    for M, want in ((J, rank_one_counts([1] * n, [1] * n)), (A, rank_one_counts(list(d), list(e)))):
        assert pf3.perm_f3_counts(M) == want
        assert _device_counts(pf3, M) == want
        if n > 32:
            assert pf3.column_merge(M) is not None
            try:
                pf3.set_class_limit(0)
                assert pf3.perm_f3_counts(M) == want
            finally:
                pf3.set_class_limit(keep)


def test_dense_terms_batch_and_ranges(pf3, oracle):
    """The batch path on dense matrices (closed form), ranges that start and
    end inside dense walks (additivity), and few-distinct-column matrices
    where only some blocks switch, against the oracle."""
    mats, want = [], []
    for k, n in enumerate([14, 18, 22, 26, 30, 33, 35]):
        A, d, e = _rank_one(7100 + k, n)
        mats.append(A)
        p, m = rank_one_counts(list(d), list(e))
        want.append(((p - m) * (-1) ** n) % 3)
    assert list(pf3.perm_f3_batch(mats)) == want
    A, _, _ = _rank_one(7200, 34)
    whole = pf3.perm_f3_range_counts(A, 12345, (1 << 33) + 777)
    mid = (1 << 32) + 4321
    lo = pf3.perm_f3_range_counts(A, 12345, mid - 1)
    hi = pf3.perm_f3_range_counts(A, mid, (1 << 33) + 777)
    assert (lo[0] + hi[0], lo[1] + hi[1]) == whole
    rng = np.random.default_rng(7300)
    for n in (16, 20, 23):
        for pool in (2, 3):
            cols = rng.integers(0, 3, size=(pool, n))
            pick = rng.integers(0, pool, size=n)
            scale = rng.choice([1, 2], size=n)
            A = ((cols[pick].T * scale) % 3).astype(np.uint8)  # column j = scale_j * cols[pick_j]
            assert pf3.perm_f3_counts(A) == oracle.counts(T(A)), (n, pool)


# known answers at the benchmark sizes (n = 36, 40): closed forms and
# oracle-sized factors; every one walks all 2^n Gray indices on the GPU

@pytest.mark.parametrize("n", [33, 36, 40])
def test_known_answers_large(pf3, oracle, n):
    assert pf3.perm_f3(np.eye(n, dtype=np.uint8)) == 1
    assert pf3.perm_f3(np.ones((n, n), np.uint8)) == math.factorial(n) % 3
    st = inputs.Stream(77, n)
    M = inputs.monomial(st, n)
    expect = 1
    for v in M[M != 0]:
        expect = expect * int(v) % 3
    assert pf3.perm_f3(M) == expect
    # P1 * blockdiag(B1, B2) * P2 with two random blocks of about n/2
    a = n // 2
    B1 = inputs.uniform_matrix(5000 + n, a)
    B2 = inputs.uniform_matrix(5001 + n, n - a)
    P1, P2 = inputs.monomial(st, n), inputs.monomial(st, n)
    X = inputs.f3_matmul(inputs.f3_matmul(P1, inputs.block_diag(B1, B2)), P2)
    scale = 1
    for v in list(P1[P1 != 0]) + list(P2[P2 != 0]):
        scale = scale * int(v) % 3
    expect = oracle.perm_mod3(B1) * oracle.perm_mod3(B2) * scale % 3
    assert pf3.perm_f3(X) == expect


@pytest.mark.parametrize("n", [36, 40])
def test_config_sizes_invariances(pf3, n):
    """The benchmark matrices at full size: properties that hold at any n."""
    seed = inputs.SEED_N36 if n == 36 else inputs.SEED_N40
    A = inputs.uniform_matrix(seed, n)
    p = pf3.perm_f3(A)
    assert p in (0, 1, 2)
    assert pf3.perm_f3(T(A)) == p
    rng = np.random.default_rng(n)
    assert pf3.perm_f3(A[rng.permutation(n)][:, rng.permutation(n)].copy()) == p
    S = A.copy()
    S[3] = (2 * S[3].astype(np.int64) % 3).astype(np.uint8)
    assert pf3.perm_f3(S) == (2 * p) % 3


@pytest.mark.parametrize("n", [36, 48])
def test_config_sizes_sampled_ranges(pf3, oracle, n):
    """Full-size benchmark matrices: sampled Gray ranges, one by one."""
    seed = inputs.SEED_N36 if n == 36 else inputs.SEED_N48
    A = inputs.uniform_matrix(seed, n)
    At = T(A)
    rng = np.random.default_rng(1 + n)
    top = (1 << n) - 1
    for _ in range(8):
        a = int(rng.integers(0, top - (1 << 18)))
        b = a + int(rng.integers(1 << 16, 1 << 18))
        assert pf3.perm_f3_range_counts(A, a, b) == oracle.ryser_range_par(At, a, b)


def test_config_n48_window_with_nonzero_terms(pf3, oracle):
    """The seeded 48 x 48 matrix: a ragged window of 2^31 Gray indices, count
    for count, with the nonzero terms it must hold (about 7.5 expected)."""
    A = inputs.uniform_matrix(inputs.SEED_N48, 48)
    a = (1 << 40) + 99
    b = a + (1 << 31) + 17
    want = oracle.ryser_range_par(T(A), a, b)
    assert sum(want) >= 5, want
    assert pf3.perm_f3_range_counts(A, a, b) == want


def test_edge_cases(pf3):
    assert pf3.perm_f3(np.zeros((0, 0), np.uint8)) == 1
    assert pf3.perm_f3_counts(np.zeros((0, 0), np.uint8)) == (1, 0)
    for v in (0, 1, 2):
        assert pf3.perm_f3(np.array([[v]], np.uint8)) == v
    with pytest.raises(pf3.PF3Error) as e:
        pf3.perm_f3(np.array([[0, 3], [1, 1]], np.uint8))
    assert e.value.code == pf3.PF3_EDOMAIN
    with pytest.raises(pf3.PF3Error) as e:
        pf3.perm_f3_range_counts(np.eye(4, dtype=np.uint8), 5, 16)
    assert e.value.code == pf3.PF3_EINVAL
    with pytest.raises(pf3.PF3Error):
        pf3.perm_f3(np.zeros((65, 65), np.uint8))
    # W = 2: a zero column makes every row-subset product 0; a zero row makes
    # the terms of S and S + {row} cancel in pairs
    Z = inputs.uniform_matrix(9, 40)
    Z[:, 7] = 0
    assert pf3.perm_f3(Z) == 0
    assert pf3.perm_f3_counts(Z) == (0, 0)
    Z = inputs.uniform_matrix(10, 35)
    Z[4] = 0
    p, m = pf3.perm_f3_counts(Z)
    assert p == m and pf3.perm_f3(Z) == 0


def test_device_pointer_entry(pf3, oracle):
    import torch
    A = inputs.uniform_matrix(11, 22)
    dA = torch.from_numpy(A).cuda()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pf3.perm_f3_range_counts_async(dA, 22, 0, (1 << 22) - 1, out, s)
    s.synchronize()
    p, m, r = [int(x) for x in out.cpu()]
    assert (p, m) == oracle.counts(T(A))
    assert r == oracle.perm_mod3(A)
    bad = dA.clone()
    bad[0, 0] = 7
    with torch.cuda.stream(s):
        pf3.perm_f3_range_counts_async(bad, 22, 0, (1 << 22) - 1, out, s)
    s.synchronize()
    assert int(out[2].cpu()) == -1  # UINT64_MAX flags the bad entry
    # the scratch is clean again afterwards
    with torch.cuda.stream(s):
        pf3.perm_f3_range_counts_async(dA, 22, 0, (1 << 22) - 1, out, s)
    s.synchronize()
    assert int(out[2].cpu()) == r


# ------------------------------------------------------------ batches

def test_batch_uniform_n24_sample(pf3, oracle):
    mats = list(inputs.uniform_matrices(inputs.SEED_BATCH24, 24, 24))
    res, hist = pf3.perm_f3_batch(mats, with_hist=True)
    want = oracle.perm_batch(mats)
    assert list(res) == list(want)
    assert list(hist) == [int((want == v).sum()) for v in range(3)]


def test_batch_mixed_sizes(pf3, oracle):
    rng = np.random.default_rng(8)
    ns = [0, 1, 2, 3, 5, 7, 8, 9, 12, 16, 20, 22] + [int(x) for x in rng.integers(1, 23, 40)]
    mats = [inputs.uniform_matrix(6000 + k, n) for k, n in enumerate(ns)]
    res = pf3.perm_f3_batch(mats)
    want = [1 if n == 0 else oracle.perm_mod3(M) for n, M in zip(ns, mats)]
    assert list(res) == want


def test_batch_single_vs_batch_identity(pf3):
    """The same matrices alone and in a mixed batch (including split items)."""
    ns = [36, 30, 29, 24, 13, 40]
    mats = [inputs.uniform_matrix(7000 + k, n) for k, n in enumerate(ns)]
    alone = [pf3.perm_f3(M) for M in mats]
    assert list(pf3.perm_f3_batch(mats)) == alone


def test_batch_bad_entry_and_empty(pf3):
    mats = [np.eye(3, dtype=np.uint8), np.full((2, 2), 4, np.uint8)]
    with pytest.raises(pf3.PF3Error) as e:
        pf3.perm_f3_batch(mats)
    assert e.value.code == pf3.PF3_EDOMAIN
    assert len(pf3.perm_f3_batch([])) == 0


# ------------------------------------------------------------ every variant

def test_every_single_variant(pf3, oracle):
    """Each compiled variant of the walk gives the same exact counts."""
    keep = {W: pf3.get_variant(pf3.SINGLE, W) for W in (1, 2)}
    try:
        cases = [(n, inputs.uniform_matrix(8000 + n, n)) for n in (9, 17, 24, 33, 37)]
        rng = np.random.default_rng(3)
        for v in range(pf3.variant_count(pf3.SINGLE)):
            for W in (1, 2):
                pf3.set_variant(pf3.SINGLE, W, v)
            for n, A in cases:
                if n <= 24:
                    assert pf3.perm_f3_counts(A) == oracle.counts(T(A)), (v, n)
                top = (1 << n) - 1
                a = int(rng.integers(0, max(1, top - 65537)))
                b = min(top, a + 65537)
                assert pf3.perm_f3_range_counts(A, a, b) == oracle.ryser_range(T(A), a, b), (v, n)
    finally:
        for W in (1, 2):
            pf3.set_variant(pf3.SINGLE, W, keep[W])


def test_every_batch_variant(pf3, oracle):
    keep = {W: pf3.get_variant(pf3.BATCH, W) for W in (1, 2)}
    keep_tuning = pf3.get_batch_tuning()
    try:
        ns = [5, 9, 13, 17, 20, 22, 3, 12]
        mats = [inputs.uniform_matrix(8100 + k, n) for k, n in enumerate(ns)]
        want = [oracle.perm_mod3(M) for M in mats]
        big = [inputs.uniform_matrix(8200 + k, n) for k, n in enumerate((33, 35))]
        pf3.set_batch_split(28, 20)  # split the W = 2 matrices into many items
        want_big = [pf3.perm_f3(M) for M in big]
        for v in range(pf3.variant_count(pf3.BATCH)):
            for W in (1, 2):
                pf3.set_variant(pf3.BATCH, W, v)
            assert list(pf3.perm_f3_batch(mats)) == want, v
            assert list(pf3.perm_f3_batch(big)) == want_big, v
    finally:
        pf3.set_batch_tuning(*keep_tuning.values())
        for W in (1, 2):
            pf3.set_variant(pf3.BATCH, W, keep[W])


def test_batch_packing_cutoff_and_split_modes(pf3, oracle):
    """Every packing cutoff 0..16 and every split mode (fixed, automatic at
    1..32 items per warp) gives the oracle's results on a mixed batch whose
    small sizes straddle the cutoffs and whose large ones get split."""
    keep = pf3.get_batch_tuning()
    rng = np.random.default_rng(41)
    ns = [int(x) for x in rng.integers(0, 17, size=300)] + [16] * 40 + [11] * 33 + [20, 23, 26, 29, 33, 35]
    mats = [inputs.uniform_matrix(9400 + k, n) for k, n in enumerate(ns)]
    want = [oracle.perm_mod3(M) if M.shape[0] <= 24 else None for M in mats]
    for k, M in enumerate(mats):
        if want[k] is None:
            want[k] = pf3.perm_f3(M)
    try:
        for tiny in range(0, 17):
            pf3.set_batch_tuning(tiny, 28, 0, 8)
            assert list(pf3.perm_f3_batch(mats)) == want, tiny
        for mode in ((28, 22), (20, 20), (0, 0)):
            for g in (1, 4, 32):
                pf3.set_batch_tuning(10, mode[0], mode[1], g)
                assert list(pf3.perm_f3_batch(mats)) == want, (mode, g)
    finally:
        pf3.set_batch_tuning(*keep.values())


def test_autotune_keeps_results(pf3, oracle):
    rep = pf3.autotune()
    assert all(t > 0 for t in rep["single_ms"][1] + rep["single_ms"][2])
    bt = rep["batch_tuning"]
    U = pf3.variant_info(pf3.BATCH, rep["batch_variant"][1])["U"]
    assert min(U, 16) <= bt["tiny_cutoff"] <= 16 and bt["chunk_log2"] == 0
    assert bt["items_per_warp"] in (1, 2, 4, 8, 16) and all(t > 0 for t in rep["split_ms"].values())
    # the cutoff is the last n (counting up) at which the packed walk won
    for n, (packed, warp) in rep["pack_ms"].items():
        assert (packed < warp) == (n <= bt["tiny_cutoff"]), (n, packed, warp, bt)
    A = inputs.uniform_matrix(8300, 21)
    assert pf3.perm_f3_counts(A) == oracle.counts(T(A))


def test_batch_async_graph_replay(pf3, oracle):
    """Second identical call replays the captured graph and sees new matrix
    contents; a different size list re-plans."""
    import torch
    n, count = 14, 64
    A = inputs.uniform_matrices(9100, n, count)
    B = inputs.uniform_matrices(9101, n, count)
    ns = np.full(count, n, np.int32)
    dAs = torch.from_numpy(A.reshape(-1).copy()).cuda()
    res = torch.zeros(count, dtype=torch.uint8, device="cuda")
    hist = torch.zeros(3, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    want_a = oracle.perm_batch(list(A))
    want_b = oracle.perm_batch(list(B))
    for _ in range(2):
        pf3.perm_f3_batch_async(dAs, ns, res, hist, s)
        s.synchronize()
        assert res.cpu().numpy().tolist() == want_a.tolist()
    dAs.copy_(torch.from_numpy(B.reshape(-1).copy()).cuda())
    pf3.perm_f3_batch_async(dAs, ns, res, hist, s)
    s.synchronize()
    assert res.cpu().numpy().tolist() == want_b.tolist()
    assert hist.cpu().tolist() == [int((want_b == v).sum()) for v in range(3)]
    ns2 = np.full(count // 2, n, np.int32)
    pf3.perm_f3_batch_async(dAs, ns2, res, hist, s)
    s.synchronize()
    assert res[:count // 2].cpu().numpy().tolist() == want_b[:count // 2].tolist()


def test_autotune_cache_roundtrip(tmp_path):
    """The tuned choice is written to PF3_TUNE_CACHE and loaded by a new process."""
    import os
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, PF3_TUNE_CACHE=str(cache))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2407_20205_gb300 import binding as b\n"
            "r = b.autotune()\n"
            "t = r['batch_tuning']\n"
            "print(r['single_variant'][1], r['single_variant'][2], r['batch_variant'][1], r['batch_variant'][2],"
            " t['tiny_cutoff'], t['items_per_warp'], r['single_short_variant'][1], r['single_short_variant'][2],"
            " r['single_merged_variant'])\n"
            ) % root
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    line = cache.read_text().strip().splitlines()[-1]
    assert line.split("|")[-9:] == first.stdout.split()
    code2 = ("import sys; sys.path.insert(0, %r)\n"
             "from paper_2407_20205_gb300 import binding as b\n"
             "t = b.get_batch_tuning()\n"
             "print(b.get_variant(0, 1), b.get_variant(0, 2), b.get_variant(1, 1), b.get_variant(1, 2),"
             " t['tiny_cutoff'], t['items_per_warp'], b.get_variant(2, 1), b.get_variant(2, 2), b.get_variant(3, 1))\n"
             ) % root
    second = subprocess.run([sys.executable, "-c", code2], env=env, capture_output=True, text=True, check=True)
    assert second.stdout.split() == first.stdout.split()


def test_async_calls_on_different_streams_do_not_race(pf3, oracle):
    """Two device-pointer calls on two streams and a host-pointer call, issued
    back to back with no synchronisation between them, share the device's
    scratch; the library orders them, so each result is the oracle's."""
    import torch
    mats = [inputs.uniform_matrix(12000 + k, n) for k, n in enumerate((24, 26, 33))]
    ranges = [(0, (1 << 24) - 1), (12345, (1 << 26) - 3), (777, 777 + (1 << 28))]
    want = [oracle.ryser_range_par(T(M), a, b) for M, (a, b) in zip(mats, ranges)]
    assert all(sum(w) > 0 for w in want)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    dA = [torch.from_numpy(M).cuda() for M in mats[:2]]
    torch.cuda.synchronize()
    for rep in range(3):
        outs = [torch.full((3,), 7 + rep, dtype=torch.int64, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        pf3.perm_f3_range_counts_async(dA[0], 24, *ranges[0], outs[0], s1)
        pf3.perm_f3_range_counts_async(dA[1], 26, *ranges[1], outs[1], s2)
        host = pf3.perm_f3_range_counts(mats[2], *ranges[2])
        torch.cuda.synchronize()
        for k in range(2):
            assert tuple(int(x) for x in outs[k][:2].cpu()) == want[k], (rep, k)
        assert host == want[2], rep

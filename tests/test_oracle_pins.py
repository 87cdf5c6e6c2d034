"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

None of these checks re-derives the oracle's own formula: they use closed
forms (n!, derangement numbers, products of diagonals), the paper's printed
Table 2 and Table 3, invariances of the permanent, and brute-force
enumeration on tiny inputs.  A dropped term, a wrong sign (the (-1)^n of
Eq. (2)), a wrong Gray index or a transposed operand fails at least one.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import rank_one_counts, read_golden
from paper_2407_20205_gb300 import inputs

RNG_SEED = 20240729


def f3(x):
    return int(x) % 3


def rand_mats(n, count, seed=RNG_SEED):
    return inputs.uniform_matrices(seed, n, count)


# ---------------------------------------------------------------- Eq. (1)

def test_bruteforce_closed_forms(oracle):
    for n in range(1, 10):
        # J_n: perm = n!
        assert oracle.perm_bruteforce_int(np.ones((n, n), np.uint8)) == math.factorial(n)
        # identity: 1
        assert oracle.perm_bruteforce_int(np.eye(n, dtype=np.uint8)) == 1
    # J_n - I: the derangement numbers D_n (textbook closed form)
    D = [1, 0, 1, 2, 9, 44, 265, 1854, 14833, 133496]
    for n in range(1, 10):
        M = np.ones((n, n), np.uint8) - np.eye(n, dtype=np.uint8)
        assert oracle.perm_bruteforce_int(M) == D[n]


def test_bruteforce_two_by_two_and_triangular(oracle):
    vals = [0, 1, 2]
    c = {0: 0, 1: 1, 2: -1}
    for a, b, cc, d in itertools.product(vals, repeat=4):
        M = np.array([[a, b], [cc, d]], np.uint8)
        assert oracle.perm_bruteforce_int(M) == c[a] * c[d] + c[b] * c[cc]
    rng = np.random.default_rng(1)
    for n in range(1, 9):
        for _ in range(10):
            M = np.triu(rng.integers(0, 3, (n, n))).astype(np.uint8)
            expect = 1
            for i in range(n):
                expect *= c[int(M[i, i])]
            assert oracle.perm_bruteforce_int(M) == expect
            assert oracle.perm_bruteforce_int(M.T.copy()) == expect


# ---------------------------------------------------------------- Eq. (2)

@pytest.mark.parametrize("n", list(range(1, 9)))
def test_ryser_matches_bruteforce(oracle, n):
    mats = rand_mats(n, 120 if n <= 6 else 40, seed=RNG_SEED + n)
    nonzero_odd = 0
    for M in mats:
        bf = oracle.perm_bruteforce(M)
        assert oracle.perm_mod3(M) == bf
        if n % 2 == 1 and bf != 0:
            nonzero_odd += 1
    if n % 2 == 1:
        # an odd-n matrix with nonzero permanent catches a (-1)^n sign slip
        assert nonzero_odd > 0


def test_ryser_special_cases(oracle):
    for n in range(1, 17):
        J = np.ones((n, n), np.uint8)
        assert oracle.perm_mod3(J) == math.factorial(n) % 3
        assert oracle.perm_mod3(np.eye(n, dtype=np.uint8)) == 1
        Z = rand_mats(n, 1, seed=7 + n)[0].copy()
        Z[n // 2, :] = 0
        assert oracle.perm_mod3(Z) == 0
        Z = rand_mats(n, 1, seed=70 + n)[0].copy()
        Z[:, n // 3] = 0
        assert oracle.perm_mod3(Z) == 0


def test_monomial_matrices(oracle):
    for n in range(1, 17):
        for k in range(6):
            st = inputs.Stream(555 + n, k)
            M = inputs.monomial(st, n)
            expect = 1
            for v in M[M != 0]:
                expect = expect * (1 if v == 1 else 2) % 3
            assert oracle.perm_mod3(M) == expect


def test_block_diagonal_product(oracle):
    for (a, b) in [(3, 4), (5, 6), (7, 7), (2, 11), (8, 8)]:
        for k in range(4):
            B1 = rand_mats(a, 1, seed=900 + 10 * a + k)[0]
            B2 = rand_mats(b, 1, seed=901 + 10 * b + k)[0]
            M = inputs.block_diag(B1, B2)
            expect = oracle.perm_mod3(B1) * oracle.perm_mod3(B2) % 3
            assert oracle.perm_mod3(M) == expect


@pytest.mark.parametrize("n", [5, 9, 12, 14])
def test_invariances(oracle, n):
    rng = np.random.default_rng(n)
    for M in rand_mats(n, 6, seed=300 + n):
        p = oracle.perm_mod3(M)
        # transpose (Eq. (2) sums column subsets; the paper's code sums rows)
        assert oracle.perm_mod3(M.T.copy()) == p
        # row and column permutations
        assert oracle.perm_mod3(M[rng.permutation(n)]) == p
        assert oracle.perm_mod3(M[:, rng.permutation(n)].copy()) == p
        # scaling one row by 2 (== negating it, Sec. 4's bijection) negates perm
        r = int(rng.integers(n))
        S = M.copy()
        S[r] = (2 * S[r].astype(np.int64) % 3).astype(np.uint8)
        assert oracle.perm_mod3(S) == (2 * p) % 3
        # scaling a column by 2
        c = int(rng.integers(n))
        S = M.copy()
        S[:, c] = (2 * S[:, c].astype(np.int64) % 3).astype(np.uint8)
        assert oracle.perm_mod3(S) == (2 * p) % 3


def _direct_term(M, i):
    """Brute force: the Ryser term of the column subset gray(i)."""
    n = M.shape[0]
    g = i ^ (i >> 1)
    cols = [j for j in range(n) if (g >> j) & 1]
    c = M.astype(np.int64)
    c[c == 2] = -1
    prod = 1
    for r in range(n):
        prod *= int(sum(c[r, j] for j in cols)) % 3
    prod %= 3
    sign = -1 if len(cols) % 2 else 1
    return (sign * prod) % 3  # 0, 1 or 2 (2 == -1)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14])
def test_rank_one_closed_form(oracle, n):
    """A_ij = d_i e_j with d, e in {1, -1}: every row-subset sum is e_j times
    t = sum_{i in S} d_i, so the exact +1/-1 term counts follow from
    binomial coefficients (rank_one_counts).  Two thirds of these terms are
    nonzero, unlike a random matrix's (2/3)^n.  The oracle walks column
    subsets, so it is given A^T."""
    rng = np.random.default_rng(900 + n)
    for _ in range(3):
        d = rng.choice([1, -1], size=n)
        e = rng.choice([1, -1], size=n)
        A = (np.outer(d, e) % 3).astype(np.uint8)
        assert oracle.counts(np.ascontiguousarray(A.T)) == rank_one_counts(list(d), list(e))
    J = np.ones((n, n), np.uint8)
    assert oracle.counts(J) == rank_one_counts([1] * n, [1] * n)


def test_range_single_index_terms(oracle):
    for n in (1, 3, 6, 9):
        M = rand_mats(n, 1, seed=40 + n)[0]
        for i in range(1 << n):
            p, m = oracle.ryser_range(M, i, i)
            t = _direct_term(M, i)
            assert (p, m) == ((1, 0) if t == 1 else (0, 1) if t == 2 else (0, 0))


def test_range_partition_sums(oracle):
    rng = np.random.default_rng(3)
    for n in (10, 13, 17):
        M = rand_mats(n, 1, seed=60 + n)[0]
        last = (1 << n) - 1
        whole = oracle.ryser_range(M, 0, last)
        cuts = sorted(set(int(x) for x in rng.integers(1, last, 7)))
        bounds = [0] + cuts + [last + 1]
        tot = [0, 0]
        for a, b in zip(bounds[:-1], bounds[1:]):
            p, m = oracle.ryser_range(M, a, b - 1)
            tot[0] += p
            tot[1] += m
        assert tuple(tot) == whole
        assert oracle.ryser_range_par(M, 0, last, nparts=13) == whole
        assert oracle.perm_from_counts(n, *whole) == oracle.perm_mod3(M)


def test_n64_range_end(oracle):
    # the last Gray index of a 64 x 64 matrix is 2^64 - 1: the inclusive bound
    M = rand_mats(64, 1, seed=64)[0]
    last = (1 << 64) - 1
    p, m = oracle.ryser_range(M, last - 300, last)
    q = oracle.ryser_range(M, last - 300, last - 101)
    r = oracle.ryser_range(M, last - 100, last)
    assert (p, m) == (q[0] + r[0], q[1] + r[1])
    # a zero column forces every term to zero
    Z = M.copy()
    Z[:, 5] = 0
    assert oracle.ryser_range(Z, last - 50, last) == (0, 0)


def test_edge_sizes(oracle):
    assert oracle.perm_mod3(np.zeros((0, 0), np.uint8)) == 1
    for v in (0, 1, 2):
        assert oracle.perm_mod3(np.array([[v]], np.uint8)) == v
        assert oracle.perm_bruteforce(np.array([[v]], np.uint8)) == v
    with pytest.raises(ValueError):
        oracle.perm_mod3(np.array([[3]], np.uint8))


# ------------------------------------------------------------ Table 2

def test_table2_exhaustive_small(oracle):
    rows = {int(r[0]): int(r[1]) for r in read_golden("table2_zn.txt")}
    for n in (1, 2, 3):
        z, c1, c2 = oracle.count_exhaustive(n)
        assert z == rows[n]
        assert c1 == c2  # the row-negation bijection of Sec. 4
        assert z + c1 + c2 == 3 ** (n * n)


def test_table2_exhaustive_n4(oracle):
    rows = {int(r[0]): int(r[1]) for r in read_golden("table2_zn.txt")}
    z, c1, c2 = oracle.count_exhaustive(4)
    assert z == rows[4] == 17116353
    assert c1 == c2
    assert z + c1 + c2 == 3 ** 16


# ------------------------------------------------------------ Table 3

@pytest.mark.parametrize("n,trials", [(6, 60000), (7, 40000)])
def test_table3_monte_carlo(oracle, n, trials):
    rows = {int(r[0]): (int(r[1]), int(r[2])) for r in read_golden("table3_montecarlo.txt")}
    zc, lg = rows[n]
    p_paper = zc / 10 ** lg
    mats = inputs.uniform_matrices(7000 + n, n, trials)
    res = oracle.perm_batch(list(mats))
    zeros = int((res == 0).sum())
    sd = math.sqrt(p_paper * (1 - p_paper) / trials)
    assert abs(zeros / trials - p_paper) < 4.5 * sd
    # and distinguishable from 1/3 (the paper's point for small n)
    assert abs(zeros / trials - 1 / 3) > 4 * sd
    c1 = int((res == 1).sum())
    c2 = int((res == 2).sum())
    assert abs(c1 - c2) < 5 * math.sqrt(trials)


# ------------------------------------------------------------ generator

def test_generator_vectorised_matches_scalar():
    for n in (1, 5, 24, 36):
        for k in (0, 3, 17):
            a = inputs.uniform_matrices(99, n, 1, start=k)[0]
            b = inputs.uniform_matrix_from_stream(inputs.Stream(99, k), n)
            assert np.array_equal(a, b)
    A = inputs.uniform_matrices(24, 24, 40)
    assert A.shape == (40, 24, 24) and A.max() <= 2
    frac = np.bincount(A.ravel(), minlength=3) / A.size
    assert np.all(np.abs(frac - 1 / 3) < 0.02)


def test_splitmix_reference_values():
    # splitmix64 from state 0: published first outputs of the reference
    # implementation (seed 0): 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4
    st = inputs.Stream(0, 0)
    st.state = 0
    assert st.next() == 0xE220A8397B1DCDAF
    assert st.next() == 0x6E789E6AA1B965F4

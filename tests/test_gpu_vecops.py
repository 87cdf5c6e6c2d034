"""The bipedal vector library (Sec. 2, Theorem 2.1): sum, difference,
pointwise product and quotient of F3 vectors, checked against F3 arithmetic on
the decoded values, exhaustively per column and on random vectors, including
the alternative zero representation (0, 1) as input."""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    return binding


def psi(m, s):
    return 0 if m == 0 else (1 if s == 0 else 2)


def test_theorem_2_1_all_sixteen_inputs(pf3):
    cases = list(itertools.product((0, 1), repeat=4))  # (m1, s1, m2, s2) per column
    # one vector per op, each of the 16 cases in its own column
    m1 = np.array([sum(c[0] << j for j, c in enumerate(cases))], np.uint64)
    s1 = np.array([sum(c[1] << j for j, c in enumerate(cases))], np.uint64)
    m2 = np.array([sum(c[2] << j for j, c in enumerate(cases))], np.uint64)
    s2 = np.array([sum(c[3] << j for j, c in enumerate(cases))], np.uint64)
    for op, f in ((pf3.OP_ADD, lambda a, b: (a + b) % 3), (pf3.OP_SUB, lambda a, b: (a - b) % 3),
                  (pf3.OP_MUL, lambda a, b: (a * b) % 3)):
        m3, s3 = pf3.vec_op(op, 16, m1, s1, m2, s2)
        for j, (a1, b1, a2, b2) in enumerate(cases):
            got = psi((int(m3[0]) >> j) & 1, (int(s3[0]) >> j) & 1)
            assert got == f(psi(a1, b1), psi(a2, b2)), (op, j)
    m3, s3 = pf3.vec_op(pf3.OP_DIV, 16, m1, s1, m2, s2)
    for j, (a1, b1, a2, b2) in enumerate(cases):
        if psi(a2, b2) == 0:
            continue  # division by zero is not defined
        a, b = psi(a1, b1), psi(a2, b2)
        want = (a * b) % 3  # b^{-1} = b in F3
        assert psi((int(m3[0]) >> j) & 1, (int(s3[0]) >> j) & 1) == want


def test_table1_exact_bits_of_the_sum(pf3):
    from conftest import read_golden
    for row in read_golden("table1_addition.txt"):
        a, b, m1, s1, m2, s2, mp, sp, free = map(int, row)
        m3, s3 = pf3.vec_op(pf3.OP_ADD, 1, [m1], [s1], [m2], [s2])
        assert (int(m3[0]), int(s3[0])) == (mp, sp)  # the theorem's own outputs, red ones included


def test_random_vectors_and_psi(pf3):
    rng = np.random.default_rng(9)
    n, count = 64, 4000
    A = rng.integers(0, 3, (count, n))
    B = rng.integers(0, 3, (count, n))

    def enc(X):
        w = np.uint64(1) << np.arange(n, dtype=np.uint64)
        mag = ((X != 0).astype(np.uint64) * w).sum(axis=1).astype(np.uint64)
        sgn = ((X == 2).astype(np.uint64) * w).sum(axis=1).astype(np.uint64)
        return mag, sgn

    ma, sa = enc(A)
    mb, sb = enc(B)
    assert np.array_equal(pf3.vec_unpack(n, ma, sa), A.astype(np.uint8))
    for op, f in ((pf3.OP_ADD, lambda x, y: (x + y) % 3), (pf3.OP_SUB, lambda x, y: (x - y) % 3),
                  (pf3.OP_MUL, lambda x, y: (x * y) % 3)):
        m3, s3 = pf3.vec_op(op, n, ma, sa, mb, sb)
        assert np.array_equal(pf3.vec_unpack(n, m3, s3), f(A, B).astype(np.uint8))


def _enc_words(X, zero_alt=None):
    """Test-side encoding of rows of X (entries 0..2) into ceil(n/64)-word
    planes, column j in bit j % 64 of word j // 64; where zero_alt is set,
    a 0 entry is written as (mag, sgn) = (0, 1)."""
    count, n = X.shape
    w = (n + 63) // 64
    mag = np.zeros((count, w), np.uint64)
    sgn = np.zeros((count, w), np.uint64)
    for j in range(n):
        bit = np.uint64(1) << np.uint64(j % 64)
        mag[:, j // 64] |= np.where(X[:, j] != 0, bit, np.uint64(0))
        s = (X[:, j] == 2) if zero_alt is None else ((X[:, j] == 2) | ((X[:, j] == 0) & zero_alt[:, j]))
        sgn[:, j // 64] |= np.where(s, bit, np.uint64(0))
    return mag, sgn


def _dec_words(mag, sgn, n):
    count = mag.shape[0]
    out = np.zeros((count, n), np.int64)
    for j in range(n):
        m = (mag[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)
        s = (sgn[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)
        out[:, j] = np.where(m == 0, 0, np.where(s == 0, 1, 2))
    return out


@pytest.mark.parametrize("n", [65, 128, 200])
def test_multiword_vectors_against_f3(pf3, n):
    """Vectors longer than 64 entries, ceil(n/64) words per plane: sum,
    difference, product and quotient against F3 arithmetic column by column,
    with inputs that use the (0, 1) zero representation, padding bits cleared
    in the results, and phi / psi round trips."""
    rng = np.random.default_rng(n)
    count = 300
    A = rng.integers(0, 3, (count, n))
    B = rng.integers(0, 3, (count, n))
    ma, sa = _enc_words(A, zero_alt=rng.random((count, n)) < 0.5)
    mb, sb = _enc_words(B, zero_alt=rng.random((count, n)) < 0.5)
    w = (n + 63) // 64
    pad = (~np.uint64(0)) << np.uint64(n % 64) if n % 64 else np.uint64(0)
    for op, f in ((pf3.OP_ADD, lambda x, y: (x + y) % 3), (pf3.OP_SUB, lambda x, y: (x - y) % 3),
                  (pf3.OP_MUL, lambda x, y: (x * y) % 3), (pf3.OP_DIV, lambda x, y: (x * y) % 3)):
        m3, s3 = pf3.vec_op(op, n, ma, sa, mb, sb)
        assert m3.shape == (count, w)
        got = _dec_words(m3, s3, n)
        want = f(A, B)
        if op == pf3.OP_DIV:
            keep = B != 0  # the quotient is defined where the divisor is nonzero
            assert np.array_equal(got[keep], want[keep])
        else:
            assert np.array_equal(got, want), op
        assert not (m3[:, -1] & pad).any() and not (s3[:, -1] & pad).any()
        assert np.array_equal(pf3.vec_unpack(n, m3, s3), got.astype(np.uint8))
    pm, ps = pf3.vec_pack(A.astype(np.uint8))
    assert np.array_equal(pm, _enc_words(A)[0]) and np.array_equal(ps, _enc_words(A)[1])
    assert np.array_equal(pf3.vec_unpack(n, pm, ps), A.astype(np.uint8))


def test_vec_pack_rejects_bad_entries_and_sizes(pf3):
    X = np.zeros((2, 70), np.uint8)
    X[1, 66] = 3
    with pytest.raises(pf3.PF3Error) as e:
        pf3.vec_pack(X)
    assert e.value.code == pf3.PF3_EDOMAIN
    with pytest.raises(ValueError):
        pf3.vec_op(pf3.OP_ADD, 70, np.zeros(3, np.uint64), np.zeros(3, np.uint64), np.zeros(3, np.uint64),
                   np.zeros(3, np.uint64))

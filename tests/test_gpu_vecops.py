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

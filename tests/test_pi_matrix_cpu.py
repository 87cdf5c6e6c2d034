"""Digits of pi for the Pi_n matrix of Sec. 3.1, pinned by an independent
algorithm (Gauss-Legendre in integer arithmetic) and by the Feynman point."""
import math

import numpy as np

from paper_2407_20205_gb300 import pi_matrix


def pi_gauss_legendre(count):
    guard = 30
    one = 10 ** (count + guard)
    a, b, t, p = one, math.isqrt(one * one // 2), one // 4, 1
    for _ in range(int(math.log2(count)) + 4):
        an = (a + b) // 2
        b = math.isqrt(a * b)
        t -= p * (a - an) ** 2 // one
        a, p = an, 2 * p
    pi = (a + b) ** 2 // (4 * t)
    return str(pi)[:count]


def test_digits_two_algorithms_agree():
    assert pi_matrix.pi_digits_machin(2600) == pi_gauss_legendre(2600)


def test_known_digits():
    d = pi_matrix.pi_digits_machin(800)
    assert d.startswith("31415926535897932384626433832795028841971693993751")
    assert d[762:768] == "999999"  # six nines from the 762nd decimal place


def test_digit_matrix_readings():
    A = pi_matrix.digit_matrix(50, "with_three")
    B = pi_matrix.digit_matrix(50, "after_point")
    d = pi_matrix.pi_digits_machin(2502)
    assert A.shape == (50, 50) and A.max() <= 2
    assert A[0, 0] == 3 % 3 and A[0, 1] == 1 and A[1, 0] == int(d[50]) % 3
    assert B[0, 0] == 1 and B[49, 49] == int(d[2500]) % 3
    assert np.array_equal(A.reshape(-1)[1:], B.reshape(-1)[:-1])

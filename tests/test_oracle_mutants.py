"""Planted mistakes in a copy of the oracle must be caught by its pins.

Each mutant is the oracle's C source with one plausible slip (a dropped sign,
a wrong Gray state, rows summed instead of columns, a wrong subtraction
direction, an off-by-one in the range walk, a wrong sign rule), compiled into
a temporary library.  The pins used here are the same facts as in
test_oracle_pins.py: brute force on small matrices, direct evaluation of single
Gray indices, Table 2 (z(3) = 8163) and partition sums.  Every mutant must fail
at least one of them, and the unmodified source must pass all of them."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from conftest import ROOT, read_golden
from paper_2407_20205_gb300 import inputs

SRC = os.path.join(ROOT, "oracle", "perm_f3_oracle.c")

MUTANTS = {
    # Eq. (2)'s (-1)^n dropped in the final map
    "no_sign_n": ("    if (n & 1) d = -d;\n    return to012(d);", "    return to012(d);"),
    # Gray state taken as i instead of i ^ (i >> 1)
    "gray_is_identity": ("uint64_t g = first ^ (first >> 1);", "uint64_t g = first;"),
    # the printed integer listing's slip: subtract when the column enters
    "enter_subtracts": ("(entering ? a[r][t] : -a[r][t])", "(entering ? -a[r][t] : a[r][t])"),
    # rows summed instead of columns (a transposed operand)
    "transposed": ("if ((g >> j) & 1u) acc += a[r][j];", "if ((g >> j) & 1u) acc += a[j][r];"),
    # the sign of a term ignores |S|
    "no_subset_sign": ("int sign = (popcount64(g) & 1) ? -1 : 1;", "int sign = 1;"),
    # the last index of a range is skipped (stops one early)
    "range_off_by_one": ("if (i == last) break;", "if (i + 1 >= last) break;"),
    # the flipped column is off by one (kept inside the matrix)
    "wrong_flip": ("int t = trailing_zeros64(i);", "int t = trailing_zeros64(i);\n        if (t > 0) t -= 1;"),
}


def build_variant(tmp_path, name, old_new):
    src = open(SRC).read()
    if old_new is not None:
        old, new = old_new
        assert old in src, f"mutation {name} does not apply"
        src = src.replace(old, new, 1)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(c), "-o", str(so)], check=True,
                   capture_output=True)
    L = ctypes.CDLL(str(so))
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.oracle_perm_bruteforce.argtypes = [u8p, ctypes.c_int]
    L.oracle_perm_mod3.argtypes = [u8p, ctypes.c_int]
    L.oracle_ryser_range.argtypes = [u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
    L.oracle_count_exhaustive.argtypes = [ctypes.c_int, ctypes.c_int, u64p]
    return L


def p8(a):
    return np.ascontiguousarray(a, dtype=np.uint8).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def direct_term(M, i):
    n = M.shape[0]
    g = i ^ (i >> 1)
    cols = [j for j in range(n) if (g >> j) & 1]
    c = M.astype(np.int64)
    c[c == 2] = -1
    prod = 1
    for r in range(n):
        prod *= int(sum(c[r, j] for j in cols)) % 3
    sign = -1 if len(cols) % 2 else 1
    return (sign * (prod % 3)) % 3


def pins_fail(L):
    """Names of the pins this library fails."""
    failed = set()
    # brute force at n = 1..6 (odd n included)
    for n in range(1, 7):
        for A in inputs.uniform_matrices(50 + n, n, 25):
            A = np.ascontiguousarray(A)
            if L.oracle_perm_mod3(p8(A), n) != L.oracle_perm_bruteforce(p8(A), n):
                failed.add("bruteforce")
                break
    # single Gray indices against direct evaluation of the subset
    M = np.ascontiguousarray(inputs.uniform_matrix(77, 6))
    for i in range(64):
        P, Q = ctypes.c_uint64(), ctypes.c_uint64()
        L.oracle_ryser_range(p8(M), 6, i, i, ctypes.byref(P), ctypes.byref(Q))
        t = direct_term(M, i)
        if (P.value, Q.value) != ((1, 0) if t == 1 else (0, 1) if t == 2 else (0, 0)):
            failed.add("single_index")
            break
    # a range split adds up to the whole
    M = np.ascontiguousarray(inputs.uniform_matrix(78, 9))
    P, Q = ctypes.c_uint64(), ctypes.c_uint64()
    L.oracle_ryser_range(p8(M), 9, 0, 511, ctypes.byref(P), ctypes.byref(Q))
    whole = (P.value, Q.value)
    tot = [0, 0]
    for a, b in ((0, 100), (101, 300), (301, 511)):
        L.oracle_ryser_range(p8(M), 9, a, b, ctypes.byref(P), ctypes.byref(Q))
        tot[0] += P.value
        tot[1] += Q.value
    if tuple(tot) != whole:
        failed.add("partition")
    # Table 2
    z = {int(r[0]): int(r[1]) for r in read_golden("table2_zn.txt")}
    c = (ctypes.c_uint64 * 3)()
    L.oracle_count_exhaustive(3, 0, c)
    if c[0] != z[3]:
        failed.add("table2")
    return failed


def test_unmodified_oracle_passes_every_pin(tmp_path):
    assert pins_fail(build_variant(tmp_path, "original", None)) == set()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    failed = pins_fail(build_variant(tmp_path, name, MUTANTS[name]))
    assert failed, f"mutant {name} passed every pin"

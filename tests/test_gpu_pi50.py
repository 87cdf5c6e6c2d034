"""perm(Pi_50) = -1 mod 3, the paper's one published permanent at n > 48
(Sec. 3.1), walked in full on the GPU: all 2^50 Gray indices in bounded
launches of 2^44 through pf3_longrun (about two and a half minutes).

The digit matrix's reading (leading 3 counted as digit 1) and its digits are
pinned on the CPU (tests/test_pi_matrix_cpu.py).  A full oracle walk of 2^50
indices does not fit a test, so the Gray window [0, 2^30) -- which holds two
nonzero terms of this matrix, found by the oracle -- is compared count for
count; its terms are asserted to be there."""
import numpy as np
import pytest

from conftest import read_golden
from paper_2407_20205_gb300 import pi_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    return binding


def test_pi50_window_vs_oracle(pf3, oracle):
    A = pi_matrix.digit_matrix(50, "with_three")
    want = oracle.ryser_range_par(np.ascontiguousarray(A.T), 0, (1 << 30) - 1)
    assert sum(want) >= 1, want
    assert pf3.perm_f3_range_counts(A, 0, (1 << 30) - 1) == want


def test_pi50_full_walk_is_minus_one(pf3):
    (n, reading, expect), = [(int(r[0]), r[1], int(r[2])) for r in read_golden("pi50_perm.txt")]
    A = pi_matrix.digit_matrix(n, reading)
    r = pf3.longrun(A, chunk_log2=pf3.LONGRUN_MAX_CHUNK_LOG2)
    assert r["finished"] and r["rc"] == 0
    assert r["plus"] + r["minus"] > 0
    assert r["perm"] == expect

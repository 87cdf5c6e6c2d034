"""Bounded launches with a checkpointed range cursor (config of the 48 x 48
long run, exercised at sizes a test can finish)."""
import os

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


def test_longrun_whole_equals_single_launch(pf3):
    A = inputs.uniform_matrix(4801, 34)
    r = pf3.longrun(A, chunk_log2=28)
    assert r["finished"] and r["rc"] == 0
    assert (r["plus"], r["minus"]) == pf3.perm_f3_counts(A)
    assert r["perm"] == pf3.perm_f3(A)


def test_longrun_interrupt_and_resume(pf3, tmp_path):
    A = inputs.uniform_matrix(4802, 33)
    ck = str(tmp_path / "ck.txt")
    first = pf3.longrun(A, chunk_log2=25, checkpoint=ck, max_seconds=1e-6)
    assert first["rc"] == pf3.PF3_ETIMEDOUT and not first["finished"]
    assert 0 < first["next_index"] < (1 << 33)
    assert os.path.exists(ck)
    # the checkpoint of this matrix is refused for another one
    with pytest.raises(pf3.PF3Error):
        pf3.longrun(inputs.uniform_matrix(4803, 33), chunk_log2=25, checkpoint=ck)
    # a cancelled call makes no progress and keeps the checkpoint
    pf3.longrun_cancel(True)
    try:
        mid = pf3.longrun(A, chunk_log2=25, checkpoint=ck)
    finally:
        pf3.longrun_cancel(False)
    assert mid["rc"] == pf3.PF3_ECANCELED and mid["next_index"] == first["next_index"]
    done = pf3.longrun(A, chunk_log2=25, checkpoint=ck)
    assert done["finished"]
    assert (done["plus"], done["minus"]) == pf3.perm_f3_counts(A)
    # calling again on a finished checkpoint returns the same totals
    again = pf3.longrun(A, chunk_log2=25, checkpoint=ck)
    assert (again["plus"], again["minus"]) == (done["plus"], done["minus"])


def test_longrun_n48_structured_known_answer_partial(pf3, oracle):
    """48 x 48 = P1 blockdiag(B1, B2) P2 with 24 x 24 blocks: the full 2^48
    walk is the long-run benchmark; here a prefix of it is checked against
    the oracle's own range walk, index by index counts."""
    st = inputs.Stream(48, 1)
    B1 = inputs.uniform_matrix(4804, 24)
    B2 = inputs.uniform_matrix(4805, 24)
    P1, P2 = inputs.monomial(st, 48), inputs.monomial(st, 48)
    X = inputs.f3_matmul(inputs.f3_matmul(P1, inputs.block_diag(B1, B2)), P2)
    r = pf3.longrun(X, chunk_log2=30, max_seconds=1e-6)
    assert not r["finished"]
    got = pf3.perm_f3_range_counts(X, 0, r["next_index"] - 1)
    assert (r["plus"], r["minus"]) == got
    want = oracle.ryser_range_par(np.ascontiguousarray(X.T), 0, (1 << 22) - 1)
    assert pf3.perm_f3_range_counts(X, 0, (1 << 22) - 1) == want


def test_n48_full_walk_known_answer(pf3, oracle):
    """The 48 x 48 size walked completely (2^48 Gray indices, bounded launches)
    on a matrix whose permanent is fixed by closed forms and two 24 x 24
    oracle permanents: perm(P1 B P2) = perm(B1) perm(B2) * (nonzero scales)."""
    st = inputs.Stream(48, 2)
    B1 = inputs.uniform_matrix(4806, 24)
    B2 = inputs.uniform_matrix(4807, 24)
    P1, P2 = inputs.monomial(st, 48), inputs.monomial(st, 48)
    X = inputs.f3_matmul(inputs.f3_matmul(P1, inputs.block_diag(B1, B2)), P2)
    scale = 1
    for v in list(P1[P1 != 0]) + list(P2[P2 != 0]):
        scale = scale * int(v) % 3
    expect = oracle.perm_mod3(B1) * oracle.perm_mod3(B2) * scale % 3
    r = pf3.longrun(X, chunk_log2=44)
    assert r["finished"] and r["perm"] == expect

"""The no-allocation range entry point (perm_f3_range_counts_noalloc).

It serves callers that must not let the library allocate device memory (a
process whose memory manager owns the whole GPU, or one that cannot afford
the device-wide synchronisation of cudaMalloc/cudaFree).  Its scratch is a
fixed array inside the library, shared by every call, so this file checks two
calls in a row against the ordinary allocating entry point (exact, integer
counts), and that an oversized request is refused.  The file is named to be
collected last; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2407_20205_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    return torch, binding


def _both(torch, pf3, A, first, last, stream):
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    ref = torch.zeros(3, dtype=torch.int64, device="cuda")
    got = torch.full((3,), 12345, dtype=torch.int64, device="cuda")
    pf3.perm_f3_range_counts_async(dA, n, first, last, ref, stream)
    pf3.perm_f3_range_counts_noalloc(dA, n, first, last, got, 0, stream)
    stream.synchronize()
    return [int(x) for x in ref.cpu()], [int(x) for x in got.cpu()]


def test_noalloc_matches_allocating_entry_two_calls(env):
    torch, pf3 = env
    s = torch.cuda.Stream()
    A = inputs.uniform_matrix(911, 27)
    B = inputs.uniform_matrix(912, 38)
    # first call (W = 1, whole range), then a second one (W = 2, ragged range)
    ref1, got1 = _both(torch, pf3, A, 0, (1 << 27) - 1, s)
    ref2, got2 = _both(torch, pf3, B, 12345, (1 << 33) + 999, s)
    assert got1 == ref1
    assert got2 == ref2
    assert got1[2] in (0, 1, 2) and got2[2] in (0, 1, 2)


def test_noalloc_matches_oracle_on_a_ragged_window(env, oracle):
    """Directly against the oracle: a ragged window (neither end on a block
    boundary) of a two-word matrix that holds nonzero terms."""
    torch, pf3 = env
    s = torch.cuda.Stream()
    A = inputs.uniform_matrix(915, 33)
    first, last = 54321, 54321 + (1 << 27) + 333
    want = oracle.ryser_range_par(np.ascontiguousarray(A.T), first, last)
    assert sum(want) > 0, want
    dA = torch.from_numpy(A).cuda()
    out = torch.full((3,), 5, dtype=torch.int64, device="cuda")
    pf3.perm_f3_range_counts_noalloc(dA, 33, first, last, out, 0, s)
    s.synchronize()
    assert tuple(int(x) for x in out[:2].cpu()) == want


def test_noalloc_limits_and_bad_entries(env):
    torch, pf3 = env
    s = torch.cuda.Stream()
    A = inputs.uniform_matrix(913, 20)
    dA = torch.from_numpy(A).cuda()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    with pytest.raises(pf3.PF3Error) as e:
        pf3.perm_f3_range_counts_noalloc(dA, 20, 0, (1 << 20) - 1, out, pf3.NOALLOC_MAX_CTAS + 1, s)
    assert e.value.code == pf3.PF3_ETOOBIG
    # an explicit small grid gives the same counts
    ref = torch.zeros(3, dtype=torch.int64, device="cuda")
    pf3.perm_f3_range_counts_async(dA, 20, 0, (1 << 20) - 1, ref, s)
    pf3.perm_f3_range_counts_noalloc(dA, 20, 0, (1 << 20) - 1, out, 3, s)
    s.synchronize()
    assert out.cpu().tolist() == ref.cpu().tolist()
    # a bad entry is reported and the shared flags are clean for the next call
    bad = dA.clone()
    bad[1, 1] = 9
    pf3.perm_f3_range_counts_noalloc(bad, 20, 0, (1 << 20) - 1, out, 0, s)
    s.synchronize()
    assert int(out[2].cpu()) == -1
    pf3.perm_f3_range_counts_noalloc(dA, 20, 0, (1 << 20) - 1, out, 0, s)
    s.synchronize()
    assert out.cpu().tolist() == ref.cpu().tolist()


def test_noalloc_small_grids_take_every_chunk_phase(env):
    """With 1, 3 or 7 CTAs a 2^31-index range is far above 512 blocks per
    lane, so the few warps run every guided phase and the tail chunks; the
    counts must equal the allocating entry point's (full grid)."""
    torch, pf3 = env
    s = torch.cuda.Stream()
    A = inputs.uniform_matrix(914, 36)
    dA = torch.from_numpy(A).cuda()
    ref = torch.zeros(3, dtype=torch.int64, device="cuda")
    first, last = 4321, (1 << 31) + 98765
    pf3.perm_f3_range_counts_async(dA, 36, first, last, ref, s)
    for ctas in (1, 3, 7):
        out = torch.full((3,), 7, dtype=torch.int64, device="cuda")
        pf3.perm_f3_range_counts_noalloc(dA, 36, first, last, out, ctas, s)
        s.synchronize()
        assert out.cpu().tolist() == ref.cpu().tolist(), ctas

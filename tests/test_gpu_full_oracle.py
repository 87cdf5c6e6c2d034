"""Opt-in (PF3_FULL_ORACLE=1): the benchmark's seeded 36 x 36 matrix walked
completely by the oracle on the host cores (2^36 Gray indices, minutes on a
16-core host) and compared exactly with the GPU's counts from the same entry
point the benchmark times.  Off by default because of the CPU time."""
import os

import numpy as np
import pytest

from paper_2407_20205_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(os.environ.get("PF3_FULL_ORACLE") != "1", reason="set PF3_FULL_ORACLE=1 (minutes of CPU)")
def test_n36_full_walk_vs_oracle(oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_20205_gb300 import binding
    A = inputs.uniform_matrix(inputs.SEED_N36, 36)
    dA = torch.from_numpy(A).cuda()
    out = torch.zeros(3, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    binding.perm_f3_range_counts_async(dA, 36, 0, (1 << 36) - 1, out, s)
    s.synchronize()
    p, m, r = [int(x) for x in out.cpu()]
    want = oracle.ryser_range_par(np.ascontiguousarray(A.T), 0, (1 << 36) - 1, nparts=4096)
    assert (p, m) == want
    assert r == oracle.perm_from_counts(36, *want)

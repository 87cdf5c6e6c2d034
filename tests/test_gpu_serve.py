"""Serving (continuous batching) on the GPU: every request's result is the same
alone and in the mix, known-answer requests match their closed forms, and the
request API reports busy / timeout / cancel / domain errors."""
import math
import time

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


def known_answer(kind, M, parts, oracle):
    n = M.shape[0]
    if kind == "ones":
        return math.factorial(n) % 3
    if kind == "perm_identity":
        r = 1
        for v in M[M != 0]:
            r = r * int(v) % 3
        return r
    if kind == "blockdiag":
        r = 1
        for B in parts["blocks"]:
            r = r * oracle.perm_mod3(B) % 3
        for P in (parts["P1"], parts["P2"]):
            for v in P[P != 0]:
                r = r * int(v) % 3
        return r
    return None


def test_mix_equals_alone(pf3, oracle):
    """Continuous batching: results in the mix equal the results alone."""
    from paper_2407_20205_gb300 import serve
    trace = serve.make_trace(inputs.SEED_SERVE, 400, 12, 30)
    arrivals = inputs.poisson_arrivals(inputs.SEED_SERVE, len(trace), 20000.0)
    res, lat, makespan, stats = serve.replay(trace, arrivals, {"chunk_log2": 18, "launch_budget": 1 << 30})
    alone = [pf3.perm_f3(A) for (n, kind, A, parts) in trace]
    assert res == alone
    assert stats["launches"] > 1 and stats["jobs_done"] >= len(trace)
    for (n, kind, A, parts), r in zip(trace, res):
        ka = known_answer(kind, A, parts, oracle)
        if ka is not None:
            assert r == ka, (n, kind)
    # a sample checked against the oracle directly
    for (n, kind, A, parts), r in list(zip(trace, res))[:40]:
        if n <= 22:
            assert r == oracle.perm_mod3(A)


def test_overlap_large_and_small(pf3):
    """Small requests that arrive while a large one runs finish first."""
    big = inputs.uniform_matrix(31, 38)
    smalls = [inputs.uniform_matrix(300 + k, 14) for k in range(50)]
    with pf3.ServeContext(chunk_log2=22) as ctx:
        tb = ctx.submit(big)
        ts = [ctx.submit(M) for M in smalls]
        rs = [ctx.wait(t) for t in ts]
        done_small = max(ctx.times(t)[1] for t in ts)
        rb = ctx.wait(tb)
        done_big = ctx.times(tb)[1]
    assert rs == [pf3.perm_f3(M) for M in smalls]
    assert rb == pf3.perm_f3(big)
    assert done_small < done_big


def test_request_api_errors(pf3):
    with pf3.ServeContext(max_jobs=1, queue_depth=2, chunk_log2=20) as ctx:
        with pytest.raises(pf3.PF3Error) as e:
            ctx.submit(np.full((3, 3), 5, np.uint8))
        assert e.value.code == pf3.PF3_EDOMAIN
        big = inputs.uniform_matrix(77, 36)
        t0 = ctx.submit(big)
        # the single slot is busy: one more waits in the queue, then the queue is full
        codes = [ctx.try_submit(np.eye(5, dtype=np.uint8)) for _ in range(4)]
        assert pf3.PF3_EBUSY in codes
        assert ctx.wait_code(t0, timeout_us=1) == pf3.PF3_ETIMEDOUT
        assert ctx.poll(t0) is None
        assert ctx.wait(t0) == pf3.perm_f3(big)
        ok = [c for c in codes if c >= 0]
        for t in ok:
            assert ctx.wait(t) == 1
        assert ctx.submit(np.zeros((0, 0), np.uint8)) >= 0


def test_cancel_queued(pf3):
    with pf3.ServeContext(max_jobs=1, chunk_log2=20) as ctx:
        t_big = ctx.submit(inputs.uniform_matrix(78, 37))
        queued = [ctx.submit(np.eye(6, dtype=np.uint8)) for _ in range(3)]
        time.sleep(0.002)  # the big request holds the only slot by now
        n = ctx.cancel_queued()
        assert n >= 1
        codes = [ctx.wait_code(t) for t in queued]
        assert codes.count(pf3.PF3_ECANCELED) == n
        assert all(c in (0, pf3.PF3_ECANCELED) for c in codes)
        assert ctx.wait(t_big) == pf3.perm_f3(inputs.uniform_matrix(78, 37))
        # the context keeps serving afterwards
        assert ctx.wait(ctx.submit(np.eye(9, dtype=np.uint8))) == 1


def test_mix_with_two_word_jobs(pf3, oracle):
    """The serving mix over its full range n = 12..40, plus two-word jobs that
    reach the batch kernel's queued replay and dense walks (first 32 columns
    drawn from a few column vectors) and two-word block-diagonal products
    with oracle-sized blocks.  Every result in the mix (the batch kernel)
    equals the single-matrix kernel's alone; every job with n <= 24 equals
    the oracle's perm; every known-answer job, the two-word block products
    among them, equals its closed form over oracle-sized factors."""
    from paper_2407_20205_gb300 import serve
    trace = serve.make_trace(inputs.SEED_SERVE + 1, 240, 12, 40)
    extra = []
    for k, (n, pool) in enumerate([(33, 2), (34, 16), (36, 3), (40, 12), (37, 2), (39, 18)]):
        extra.append((n, "pooled", inputs.pooled_columns(7700 + k, n, pool, None), None))
    st = inputs.Stream(7800, 0)
    for k, n in enumerate((34, 38, 40)):
        a = n // 2
        B1, B2 = inputs.uniform_matrix(7810 + k, a), inputs.uniform_matrix(7820 + k, n - a)
        P1, P2 = inputs.monomial(st, n), inputs.monomial(st, n)
        M = inputs.f3_matmul(inputs.f3_matmul(P1, inputs.block_diag(B1, B2)), P2)
        extra.append((n, "blockdiag", M, {"blocks": [B1, B2], "P1": P1, "P2": P2}))
    # interleave the extra jobs into the trace
    jobs = []
    for i, t in enumerate(trace):
        jobs.append(t)
        if i % 25 == 0 and extra:
            jobs.append(extra.pop(0))
    jobs.extend(extra)
    assert sum(1 for t in jobs if t[0] > 32) >= 60
    arrivals = inputs.poisson_arrivals(inputs.SEED_SERVE + 1, len(jobs), 400.0)
    res, lat, makespan, stats = serve.replay(jobs, arrivals)
    alone = [pf3.perm_f3(A) for (n, kind, A, parts) in jobs]
    assert res == alone
    checked = 0
    for (n, kind, A, parts), r in zip(jobs, res):
        ka = known_answer(kind, A, parts, oracle)
        if ka is not None:
            assert r == ka, (n, kind)
            checked += 1
        elif n <= 24:
            assert r == oracle.perm_mod3(A), (n, kind)
            checked += 1
    assert checked >= 100
    assert sum(1 for (n, kind, A, parts) in jobs if kind == "blockdiag" and n > 32) >= 3

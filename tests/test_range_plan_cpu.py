"""The single-matrix launch plan (host logic, no GPU): a Gray range [first,
last] is cut into a ragged head, whole blocks of 2^U indices and a ragged tail
that together cover it exactly once (Sec. 3.1's blocks of consecutive Gray
states); long launches hand the blocks out as guided chunks that tile them,
every chunk a multiple of 32 blocks except the last, phase lengths
non-increasing."""
import numpy as np
import pytest

from paper_2407_20205_gb300 import binding as pf3

NV = pf3.variant_count(pf3.SINGLE)


def check_cover(n, first, last, p):
    U = p["U"]
    pieces = []
    if p["has_head"]:
        pieces.append((p["head_first"], p["head_last"]))
    if p["mid_NB"]:
        pieces.append((p["mid_B0"] << U, ((p["mid_B0"] + p["mid_NB"]) << U) - 1))
    if p["has_tail"]:
        pieces.append((p["tail_first"], p["tail_last"]))
    assert pieces[0][0] == first and pieces[-1][1] == last
    for (a, b), (c, d) in zip(pieces, pieces[1:]):
        assert c == b + 1
    if p["mid_NB"]:
        # ragged ends are shorter than a block
        if p["has_head"]:
            assert p["head_last"] - p["head_first"] + 1 < (1 << U)
        if p["has_tail"]:
            assert p["tail_last"] - p["tail_first"] + 1 < (1 << U)


def check_chunks(p, grid):
    warps = grid * p["threads"] // 32
    NB = p["mid_NB"]
    assert p["dynamic"] == (1 if NB >= warps * 32 * 512 else 0)
    if not p["dynamic"]:
        assert p["chunks"] == []
        return
    pos = 0
    lens = []
    for first, ln in p["chunks"]:
        assert first == pos and ln > 0
        pos += ln
        lens.append(ln)
    assert pos == NB and len(lens) == p["nchunks"]
    assert all(x % 32 == 0 for x in lens[:-1])
    assert lens == sorted(lens, reverse=True)
    assert lens[0] <= NB // (8 * warps)            # each phase takes half of what is left
    assert min(lens[:-1] or [128]) >= 128           # the shortest chunks are 4 blocks per lane


@pytest.mark.parametrize("variant", range(NV))
def test_range_plan_random_ranges(variant):
    rng = np.random.default_rng(31 + variant)
    for n in (5, 9, 10, 17, 24, 33, 40, 48, 64):
        top = (1 << n) - 1
        for _ in range(6):
            a = int(rng.integers(0, top + 1, dtype=np.uint64)) if n < 64 else int(rng.integers(0, 2**63)) * 2
            b = int(rng.integers(a, top + 1, dtype=np.uint64)) if n < 64 else top
            for grid in (1, 7, 304):
                p = pf3.range_plan(n, a, b, variant, grid)
                check_cover(n, a, b, p)
                if p["nchunks"] < 200000:
                    check_chunks(p, grid)


def test_range_plan_whole_walks_and_threshold():
    # the benchmark sizes on the default grid: 36 x 36 and 40 x 40 take guided chunks
    for n in (36, 40):
        p = pf3.range_plan(n, 0, (1 << n) - 1, 0, 304)
        assert p["dynamic"] == 1 and not p["has_head"] and not p["has_tail"]
        assert p["mid_NB"] == 1 << (n - 9)
        check_chunks(p, 304)
    # 2^34 indices (431 blocks per lane) stays on fixed shares, 2^35 (862) does not
    assert pf3.range_plan(40, 0, (1 << 34) - 1, 0, 304)["dynamic"] == 0
    assert pf3.range_plan(40, 0, (1 << 35) - 1, 0, 304)["dynamic"] == 1
    # n <= U: one generic head walk
    p = pf3.range_plan(9, 0, 511, 0, 304)
    assert p["has_head"] and p["mid_NB"] == 0 and not p["has_tail"]
    # the top of the 64-bit index space
    p = pf3.range_plan(64, (1 << 64) - 1000, (1 << 64) - 1, 0, 304)
    check_cover(64, (1 << 64) - 1000, (1 << 64) - 1, p)


def test_range_plan_rejects_bad_arguments():
    for args in ((0, 0, 0), (65, 0, 0), (10, 5, 4), (10, 0, 1024)):
        with pytest.raises(pf3.PF3Error):
            pf3.range_plan(*args)
    with pytest.raises(pf3.PF3Error):
        pf3.range_plan(20, 0, 100, NV, 304)
    with pytest.raises(pf3.PF3Error):
        pf3.range_plan(20, 0, 100, 0, 0)

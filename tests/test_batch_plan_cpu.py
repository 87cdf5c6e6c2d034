"""The batch planner (host logic, no GPU): every matrix is covered exactly once,
split pieces tile the Gray index range (Sec. 3.1's blocks of consecutive Gray
states), packed groups hold consecutive matrices of one small n, items run
largest first, and the automatic item length follows its stated rule."""
import numpy as np
import pytest

from paper_2407_20205_gb300 import binding as pf3

U_OF = {v: pf3.variant_info(pf3.BATCH, v)["U"] for v in range(pf3.variant_count(pf3.BATCH))}


def check_cover(ns, plan, tiny, variant):
    """Each matrix appears once (packed) or its item ranges tile 2^(n-U) blocks."""
    seen = {}
    for it in plan["items"]:
        n = it["n"]
        if it["kind"] == "packed":
            assert 1 <= it["num_blocks"] <= 32 and n <= tiny and it["cls"] == 0
            for k in range(it["mat"], it["mat"] + it["num_blocks"]):
                assert ns[k] == n
                assert k not in seen
                seen[k] = "packed"
            continue
        assert n > tiny and ns[it["mat"]] == n
        U = U_OF[variant[it["cls"]]]
        assert it["cls"] == (0 if n <= 32 else 1) and it["block_log2"] == U
        if it["kind"] == "lane":
            assert n <= U and it["mat"] not in seen
            seen[it["mat"]] = "lane"
            continue
        assert n > U
        seen.setdefault(it["mat"], []).append((it["first_block"], it["num_blocks"], it["kind"]))
    assert sorted(seen) == list(range(len(ns)))
    for k, v in seen.items():
        if isinstance(v, str):
            continue
        U = U_OF[variant[0 if ns[k] <= 32 else 1]]
        v.sort()
        kinds = {x[2] for x in v}
        assert kinds == ({"whole"} if len(v) == 1 and v[0][2] == "whole" else {"piece"})
        pos = 0
        for first, nb, _ in v:
            assert first == pos and nb > 0
            pos += nb
        assert pos == 1 << (ns[k] - U)


def cost(it):
    if it["kind"] == "packed":
        return (1 << it["n"]) << 7
    if it["kind"] == "lane":
        return 1 << it["n"]
    return it["num_blocks"] << it["block_log2"]


@pytest.mark.parametrize("tiny", [0, 6, 10, 12, 16])
@pytest.mark.parametrize("mode", [(28, 0, 8), (28, 30, 8), (30, 34, 1), (0, 0, 32)])
def test_plan_covers_every_matrix(tiny, mode):
    rng = np.random.default_rng(tiny * 100 + mode[1])
    ns = [int(x) for x in rng.integers(0, 41, size=200)]
    ns += [12] * 70 + [5] * 40 + [44, 0, 1, 16, 17, 33]
    if mode[1] == 0:
        ns += [52, 64]  # the automatic split keeps these to a few thousand pieces
    variant = (0, 3)
    plan = pf3.batch_plan(ns, tiny, *mode, variant=variant, warps=(2432, 1216))
    check_cover(ns, plan, tiny, variant)
    for cls in (0, 1):
        costs = [cost(it) for it in plan["items"] if it["cls"] == cls]
        assert costs == sorted(costs, reverse=True)
    # class 1 (two words per plane) is launched first
    cls_seq = [it["cls"] for it in plan["items"]]
    assert cls_seq == sorted(cls_seq, reverse=True)


def test_packed_groups_break_at_size_changes():
    ns = [7] * 40 + [8] * 3 + [7] * 5 + [11]
    plan = pf3.batch_plan(ns, tiny_cutoff=10)
    groups = sorted((it["mat"], it["num_blocks"], it["n"]) for it in plan["items"] if it["kind"] == "packed")
    assert groups == [(0, 32, 7), (32, 8, 7), (40, 3, 8), (43, 5, 7)]
    assert [it["kind"] for it in plan["items"] if it["n"] == 11] == ["whole"]


def guided_piece_log2(ns, tiny, warps, g, U):
    """Per matrix: log2 of its piece length under the guided split (n = whole),
    from the rule as stated: largest first, the work from the matrix to the
    end of the order over warps x g, rounded down to a power of two, at least
    2^max(20, U + 5), at least 2^(n - 20)."""
    out = {}
    for cls in (0, 1):
        order = sorted((k for k, n in enumerate(ns) if n > tiny and (n <= 32) == (cls == 0)),
                       key=lambda k: -ns[k])
        rest = sum(1 << ns[k] for k in order)
        for k in order:
            n = ns[k]
            cl = max(20, U + 5)
            while (1 << (cl + 1)) * warps[cls] * g <= rest:
                cl += 1
            out[k] = n if cl >= n else max(cl, U + 5, n - 20)
            rest -= 1 << n
    return out


def test_guided_split_rule():
    warps = (2432, 1824)
    U = U_OF[0]
    for ns, g in (([28] * 600, 8), ([28] * 300 + [26] * 600 + [24] * 1200, 4), ([33] * 20 + [34] * 6, 16),
                  ([26] * 3000, 1), ([30] * 5, 2), ([20] * 10, 8), ([24, 31, 27, 40, 22] * 50, 2)):
        plan = pf3.batch_plan(ns, 10, 28, 0, g, variant=(0, 0), warps=warps)
        want = guided_piece_log2(ns, 10, warps, g, U)
        pieces = {}
        for it in plan["items"]:
            if it["kind"] in ("whole", "piece"):
                pieces.setdefault(it["mat"], []).append(it)
        for k, its in pieces.items():
            n = ns[k]
            if want[k] >= n:
                assert len(its) == 1 and its[0]["kind"] == "whole", (k, n)
            else:
                assert len(its) == 1 << (n - want[k]), (k, n, want[k], len(its))
                assert all(it["num_blocks"] << it["block_log2"] == 1 << want[k] for it in its)
        check_cover(ns, plan, 10, (0, 0))
    # pieces shrink toward the end: 3000 x 26 starts whole and ends in 2^20 pieces
    p = pf3.batch_plan([26] * 3000, items_per_warp=1, warps=(2432, 2432))
    sizes = [it["num_blocks"] << it["block_log2"] for it in p["items"]]
    assert sizes[0] == 1 << 26 and sizes[-1] == 1 << 20 and sizes == sorted(sizes, reverse=True)
    # 2,000 x 24 on a 24-warp grid (8 items per warp) is whole until fewer
    # than 24 x 8 matrices are left
    p = pf3.batch_plan([24] * 2000, warps=(24, 24))
    assert sum(it["kind"] == "whole" for it in p["items"]) == 2000 - (24 * 8 - 1)
    assert p["chunk_log2"][0] == 24


def test_fixed_split_and_item_cap():
    """Fixed mode cuts n > cutoff into 2^chunk_log2 pieces, never more than
    2^20 pieces per matrix (n = 64 uses 2^44-index pieces)."""
    plan = pf3.batch_plan([29, 28, 64], 10, 28, 20, 8)
    by = {}
    for it in plan["items"]:
        by.setdefault(it["n"], []).append(it)
    assert len(by[28]) == 1 and by[28][0]["kind"] == "whole"
    assert len(by[29]) == 1 << 9 and all(it["num_blocks"] << it["block_log2"] == 1 << 20 for it in by[29])
    assert len(by[64]) == 1 << 20
    check_cover([29, 28, 64], plan, 10, (0, 0))


def test_plan_rejects_bad_arguments():
    with pytest.raises(pf3.PF3Error):
        pf3.batch_plan([5], tiny_cutoff=17)
    with pytest.raises(pf3.PF3Error):
        pf3.batch_plan([65])
    with pytest.raises(pf3.PF3Error):
        pf3.batch_plan([5], chunk_log2=11)
    with pytest.raises(pf3.PF3Error):
        pf3.batch_plan([5], items_per_warp=0)
    with pytest.raises(pf3.PF3Error):
        pf3.batch_plan([5], warps=(0, 1))
    assert pf3.batch_plan([], warps=(1, 1))["items"] == []


def test_batch_counts_beyond_32_bit_indices_are_rejected():
    """Work items index matrices with 32-bit integers, so a count above
    PF3_MAX_BATCH (2^31 - 65) is refused before anything is read."""
    import ctypes
    va = (ctypes.c_int * 2)(0, 0)
    wa = (ctypes.c_int * 2)(2432, 2432)
    num = ctypes.c_int64()
    for count in (2**31 - 64, 2**40):
        rc = pf3._lib_plan(None, count, 10, 28, 0, 8, va, wa, None, 0, ctypes.byref(num), None)
        assert rc == pf3.PF3_EINVAL
        assert pf3._lib_batch(None, None, count, None, None) == pf3.PF3_EINVAL

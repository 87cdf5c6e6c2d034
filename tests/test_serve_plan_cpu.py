"""The serving loop's choice of work items, on the CPU (pf3_serve_plan runs the
same host functions as the scheduler: the work split of an admitted request
and the per-launch selection; no device).  The policy: every request with at
most 2^small_work_log2 Gray indices left goes first, least remaining first;
the others are served in arrival order with what is left of each launch's
budget; each request's range is cut into work items of 2^chunk_log2 indices
(Sec. 3.1's blocks of consecutive Gray states)."""
import pytest


@pytest.fixture(scope="module")
def pf3():
    from paper_2407_20205_gb300 import build
    build.build()
    from paper_2407_20205_gb300 import binding
    return binding


U = (9, 9)
CFG = dict(chunk_log2=30, launch_budget=1 << 33, launch_items=16384, small_work_log2=33)


def cost(it):
    return (1 << it["n"]) if it["num_blocks"] == 0 else it["num_blocks"] << it["block_log2"]


def plan(pf3, ns, ms=None, launches=2000, **cfg):
    c = dict(CFG, **cfg)
    items = pf3.serve_plan(ns, ms, launches=launches, U=U, **c)
    for it in items:
        it["n"] = ns[it["request"]]
    return items


def test_small_first_least_remaining_then_arrival_order(pf3):
    ns = [40, 20, 12, 36, 28, 34]
    items = plan(pf3, ns)
    first_in_launch0 = []
    for it in items:
        if it["launch"] == 0 and it["request"] not in first_in_launch0:
            first_in_launch0.append(it["request"])
    # small requests (12, 20, 28: at most 2^33 indices) by remaining work, then
    # the first large request to arrive (40)
    assert first_in_launch0[:4] == [2, 1, 4, 0]
    # large requests in arrival order: 40, then 36, then 34
    first = {r: min(i for i, it in enumerate(items) if it["request"] == r) for r in range(len(ns))}
    last = {r: max(i for i, it in enumerate(items) if it["request"] == r) for r in range(len(ns))}
    assert last[0] < first[3] and last[3] < first[5]


def test_every_request_tiles_its_range_once(pf3):
    ns = [40, 20, 12, 36, 28, 34, 9, 33]
    items = plan(pf3, ns)
    for r, n in enumerate(ns):
        mine = [it for it in items if it["request"] == r]
        if n <= U[0]:
            assert len(mine) == 1 and mine[0]["num_blocks"] == 0 and mine[0]["last"] == 1
            continue
        nb = 1 << (n - U[0])
        spans = sorted((it["first_block"], it["num_blocks"]) for it in mine)
        at = 0
        for b0, k in spans:
            assert b0 == at and k > 0
            at += k
        assert at == nb
        assert sum(it["last"] for it in mine) == 1 and mine[-1]["last"] == 1
        # items of 2^chunk_log2 indices (or at least 2^(n - 30), at most the whole range)
        want = max(CFG["chunk_log2"], U[0] + 5, n - 30)
        assert all(it["num_blocks"] << U[0] == min(1 << want, 1 << n) for it in mine[:-1])


def test_budget_and_item_cap(pf3):
    ns = [38, 26, 30, 40, 22, 35] * 3
    for budget, cap in ((1 << 33, 16384), (1 << 31, 7), (1 << 36, 100000)):
        items = plan(pf3, ns, launch_budget=budget, launch_items=cap)
        launches = {}
        for it in items:
            launches.setdefault(it["launch"], []).append(it)
        for l, its in launches.items():
            assert len(its) <= cap, l
            total = sum(cost(it) for it in its)
            # a launch keeps to its budget, except that a request's first item always goes
            assert total <= budget or len(its) == 1 or total - cost(its[-1]) < budget, (l, total)
        assert sorted(launches) == list(range(len(launches)))  # no empty launch in between


def test_all_small_is_least_remaining_first(pf3):
    ns = [30, 14, 26, 18, 22]
    items = plan(pf3, ns, small_work_log2=64, launch_budget=1 << 40)
    order = []
    for it in items:
        if it["request"] not in order:
            order.append(it["request"])
    assert order == sorted(range(len(ns)), key=lambda r: ns[r])


def test_merged_columns_take_the_one_word_class(pf3):
    items = plan(pf3, [40, 40, 36], ms=[12, 40, 33])
    cls = {it["request"]: it["cls"] for it in items}
    assert cls == {0: 0, 1: 1, 2: 1}


def test_narrow_merged_requests_are_counted_by_class(pf3):
    """A request whose merged matrix (n > 32) has at most class_max_cols
    columns gets no work items: it is counted by column-sum vector in the
    launch that admits it.  With class_max_cols = 0 it is walked."""
    ns, ms = [40, 36, 40, 20], [2, 8, 9, 20]
    items = plan(pf3, ns, ms=ms)
    assert {it["request"] for it in items} == {2, 3}
    items = plan(pf3, ns, ms=ms, class_max_cols=0)
    assert {it["request"] for it in items} == {0, 1, 2, 3}
    assert {it["cls"] for it in items if it["request"] in (0, 1)} == {0}


def test_bad_arguments(pf3):
    for ns, ms, u in (([0], None, U), ([40], [41], U), ([65], None, U), ([20], None, (0, 9)), ([20], None, (9, 21))):
        with pytest.raises(pf3.PF3Error):
            pf3.serve_plan(ns, ms, launches=1, U=u)
    with pytest.raises(pf3.PF3Error):
        pf3.serve_plan([20], launches=1, U=U, chunk_log2=5)
    for bad in (-1, pf3.CLASS_MAX_COLS + 1):
        with pytest.raises(pf3.PF3Error):
            pf3.serve_plan([20], launches=1, U=U, class_max_cols=bad)


def test_too_small_a_buffer_writes_nothing(pf3):
    import ctypes
    import numpy as np
    b = pf3
    ns = np.array([30, 35], np.int32)
    cfg = b.config_default()
    Ua = (ctypes.c_int * 2)(*U)
    num = ctypes.c_int64()
    buf = (b.ServeItem * 2)()
    for x in buf:
        x.request = -7
    rc = b._lib_serve_plan(ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, 2, ctypes.byref(cfg), Ua, 50,
                           buf, 2, ctypes.byref(num))
    assert rc == b.PF3_ETOOBIG and num.value > 2
    assert all(x.request == -7 for x in buf)

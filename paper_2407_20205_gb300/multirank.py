"""Splitting one permanent over several ranks (one process per GPU).

Sec. 3.1 of the paper runs the Gray walk as independent jobs over blocks of
consecutive Gray states and adds their partial sums.  Here each rank walks its
share of [0, 2^n) and the exact (+1, -1) counts are the only data exchanged:

* ``rank_range``    -- the contiguous share of rank r of `world`;
* ``allreduce_counts`` -- sum the two 64-bit counts over all ranks (NCCL on
  GPUs, gloo on CPUs);
* ``walk_with_recovery`` -- the same split in chunks whose results are
  published to a key-value store; rank 0 collects them and recomputes any
  chunk whose owner did not publish before the deadline (a rank that died or
  hung).  Counts are idempotent integer sums, so a recomputed chunk is exact.

``range_fn(first, last) -> (plus, minus)`` does the walking: the CUDA entry
point in production (``binding.perm_f3_range_counts``), any other exact
implementation in tests.
"""
from __future__ import annotations

import time
from typing import Callable

RangeFn = Callable[[int, int], tuple]


def rank_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Inclusive Gray-index range [first, last] of rank `rank` (may be empty:
    first > last when 2^n < world)."""
    total = 1 << n
    q, r = divmod(total, world)
    first = rank * q + min(rank, r)
    length = q + (1 if rank < r else 0)
    return first, first + length - 1


def chunks(n: int, count: int) -> list[tuple[int, int]]:
    """[0, 2^n) cut into `count` contiguous inclusive ranges (empty ones dropped)."""
    out = []
    for k in range(count):
        a, b = rank_range(n, k, count)
        if a <= b:
            out.append((a, b))
    return out


_U64 = 1 << 64


def _as_i64(x: int) -> int:
    """The int64 with the same 64 bits as the uint64 x."""
    return x - _U64 if x >= 1 << 63 else x


def allreduce_counts(plus: int, minus: int, device=None) -> tuple[int, int]:
    """Sum the two unsigned 64-bit counts over all ranks.  The collective
    works on int64, so each count travels as the int64 with the same bits; a
    two's-complement sum has the same bits as the unsigned sum mod 2^64, and
    the true total of each count is below 2^64 (at most 2^n terms), so the
    result read back as unsigned is exact even above 2^63."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([_as_i64(plus), _as_i64(minus)], dtype=torch.int64, device=device)
    dist.all_reduce(t)
    return int(t[0]) % _U64, int(t[1]) % _U64


def perm_from_counts(n: int, plus: int, minus: int) -> int:
    """perm mod 3 from the summed counts: the library's final map."""
    from . import binding
    return binding.perm_from_counts(n, plus, minus)


def walk_with_recovery(range_fn: RangeFn, n: int, rank: int, world: int, store, chunks_per_rank: int = 4,
                       deadline_s: float = 5.0, die_after: int | None = None, tag: str = "pf3") -> dict | None:
    """Chunked walk with host-side failure detection.

    Chunk k belongs to rank k % world.  Every rank walks its chunks and
    publishes "plus,minus" under key f"{tag}/chunk/{k}".  ``die_after``
    (tests only) makes this rank stop after publishing that many chunks, as if
    its process had died.  Rank 0 then waits up to ``deadline_s`` for each
    chunk and recomputes the missing ones itself.  Returns the totals on rank
    0 (with the list of recovered chunks), None on other ranks."""
    plan = chunks(n, chunks_per_rank * world)
    mine = [k for k in range(len(plan)) if k % world == rank]
    done = 0
    for k in mine:
        if die_after is not None and done >= die_after:
            break
        p, m = range_fn(*plan[k])
        store.set(f"{tag}/chunk/{k}", f"{p},{m}")
        done += 1
    if rank != 0:
        return None
    total_p = total_m = 0
    recovered = []
    t_end = time.monotonic() + deadline_s
    for k in range(len(plan)):
        key = f"{tag}/chunk/{k}"
        val = None
        while True:
            if store.check([key]):
                val = store.get(key).decode()
                break
            if time.monotonic() >= t_end:
                break
            time.sleep(0.01)
        if val is None:
            p, m = range_fn(*plan[k])
            recovered.append(k)
        else:
            p, m = (int(x) for x in val.split(","))
        total_p += p
        total_m += m
    return {"plus": total_p, "minus": total_m, "recovered": recovered, "chunks": len(plan),
            "perm": perm_from_counts(n, total_p, total_m)}

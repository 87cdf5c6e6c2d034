"""The multi-rank split (Sec. 3.1's blocks of Gray states over several jobs),
exercised with two gloo ranks on CPU.  The walking itself is the oracle's
exact range walk (on A^T: its column walk equals the kernels' row walk), so
these tests check the partition, the count reduction and the recovery of a
rank that stops, not the CUDA path."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2407_20205_gb300 import inputs, multirank


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_rank_ranges_partition():
    for n in (1, 3, 10, 17):
        for world in (1, 2, 3, 8, 13):
            parts = [multirank.rank_range(n, r, world) for r in range(world)]
            covered = []
            for a, b in parts:
                if a <= b:
                    covered.extend(range(a, b + 1))
            assert covered == list(range(1 << n))
    a, b = multirank.rank_range(64, 3, 4)
    assert (a, b) == (3 << 62, (1 << 64) - 1)


def _range_fn(A):
    import oracle
    At = np.ascontiguousarray(A.T)
    return lambda a, b: oracle.ryser_range(At, a, b)


def _worker_allreduce(rank, world, port, n, seed, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.uniform_matrix(seed, n)
    a, b = multirank.rank_range(n, rank, world)
    p, m = _range_fn(A)(a, b)
    P, M = multirank.allreduce_counts(p, m)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(f"{P} {M}")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_allreduce(tmp_path, oracle):
    n, seed = 15, 1501
    out = str(tmp_path / "res.txt")
    mp.start_processes(_worker_allreduce, args=(2, free_port(), n, seed, out), nprocs=2, start_method="spawn")
    P, M = (int(x) for x in open(out).read().split())
    A = inputs.uniform_matrix(seed, n)
    assert (P, M) == oracle.counts(np.ascontiguousarray(A.T))
    assert multirank.perm_from_counts(n, P, M) == oracle.perm_mod3(A)


def _worker_recovery(rank, world, port, n, seed, out_path, die_rank):
    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=__import__("datetime").timedelta(seconds=30))
    A = inputs.uniform_matrix(seed, n)
    res = multirank.walk_with_recovery(_range_fn(A), n, rank, world, store, chunks_per_rank=3, deadline_s=2.0,
                                       die_after=1 if rank == die_rank else None)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(f"{res['plus']} {res['minus']} {','.join(map(str, res['recovered']))}")
        # keep the store (hosted by rank 0) up until the other ranks are done
        store.wait([f"done/{r}" for r in range(1, world)])
    else:
        store.set(f"done/{rank}", "1")


def test_gloo_rank_failure_is_recovered(tmp_path, oracle):
    """Rank 1 stops after its first chunk (a failure made on the host); rank 0
    notices the missing chunks at the deadline and recomputes them."""
    n, seed = 14, 1502
    out = str(tmp_path / "res.txt")
    mp.start_processes(_worker_recovery, args=(2, free_port(), n, seed, out, 1), nprocs=2, start_method="spawn")
    fields = open(out).read().split()
    P, M = int(fields[0]), int(fields[1])
    recovered = [int(x) for x in fields[2].split(",")] if len(fields) > 2 else []
    A = inputs.uniform_matrix(seed, n)
    assert (P, M) == oracle.counts(np.ascontiguousarray(A.T))
    assert recovered == [3, 5]  # rank 1 owns chunks 1, 3, 5 and published only chunk 1


def test_gloo_three_ranks_uneven_split(tmp_path, oracle):
    """2^13 Gray indices over 3 ranks (an uneven split): the all-reduced counts
    equal the oracle's whole walk."""
    n, seed = 13, 1503
    out = str(tmp_path / "res.txt")
    mp.start_processes(_worker_allreduce, args=(3, free_port(), n, seed, out), nprocs=3, start_method="spawn")
    P, M = (int(x) for x in open(out).read().split())
    A = inputs.uniform_matrix(seed, n)
    assert (P, M) == oracle.counts(np.ascontiguousarray(A.T))


def test_gloo_three_ranks_last_rank_fails(tmp_path, oracle):
    """With 3 ranks and 3 chunks each, rank 2 owns chunks 2, 5, 8 and stops
    after publishing chunk 2; rank 0 recomputes 5 and 8 at the deadline."""
    n, seed = 14, 1504
    out = str(tmp_path / "res.txt")
    mp.start_processes(_worker_recovery, args=(3, free_port(), n, seed, out, 2), nprocs=3, start_method="spawn")
    fields = open(out).read().split()
    P, M = int(fields[0]), int(fields[1])
    recovered = [int(x) for x in fields[2].split(",")] if len(fields) > 2 else []
    A = inputs.uniform_matrix(seed, n)
    assert (P, M) == oracle.counts(np.ascontiguousarray(A.T))
    assert recovered == [5, 8]


def _worker_big_counts(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [((1 << 63) + 5, (1 << 63) - 1), ((1 << 62) + 11, 3)][rank]
    P, M = multirank.allreduce_counts(*mine)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(f"{P} {M}")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_counts_at_and_above_2_63(tmp_path, oracle):
    """Counts of 2^63 and more (reachable at n = 64) survive the int64
    collective exactly, and the library's final map of the sums agrees with
    the oracle's on them (2^64 = 1 mod 3, so a wrapped sum would not)."""
    out = str(tmp_path / "res.txt")
    mp.start_processes(_worker_big_counts, args=(2, free_port(), out), nprocs=2, start_method="spawn")
    P, M = (int(x) for x in open(out).read().split())
    assert P == (1 << 63) + 5 + (1 << 62) + 11
    assert M == (1 << 63) - 1 + 3
    for n in (63, 64):
        assert multirank.perm_from_counts(n, P, M) == oracle.perm_from_counts(n, P, M)

"""Host logic of the multi-GPU path (CPU): the length-balanced partition of
a batch and the reduction of the totals over a world-size-2 gloo group."""
import os
import socket

import numpy as np
import pytest

from paper_2202_12380_gb300 import inputs
from paper_2202_12380_gb300.shard import partition, reduce_totals


def test_partition_covers_each_signal_once_and_balances():
    lens = inputs.batch_lengths(inputs.WORKLOADS["batch256"], inputs.WORKLOADS["batch256"]["id"])
    for n in (1, 2, 3, 4, 8):
        parts = partition(lens, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(lens)))
        loads = [sum(lens[i] for i in p) for p in parts]
        # greedy longest-first: the spread is at most one signal
        assert max(loads) - min(loads) <= max(lens)
        assert parts == partition(lens, n)  # deterministic


def test_partition_edge_cases():
    assert partition([], 2) == [[], []]
    assert partition([5], 3) == [[0], [], []]
    assert partition([4, 4, 4, 4], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        partition([1], 0)


def test_reduce_totals_without_group_is_identity():
    assert reduce_totals(1.5, 7) == (1.5, 7.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, lens, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = partition(lens, world)[rank]
        # each rank "decomposes" its shard: atoms = its signals' lengths / 100,
        # time = its load in milliseconds (stand-ins computed on the host)
        atoms = sum(lens[i] // 100 for i in mine)
        secs = sum(lens[i] for i in mine) / 1e6
        t, a = reduce_totals(secs, atoms)
        q.put((rank, mine, t, a))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shards_and_totals():
    import torch.multiprocessing as mp

    lens = [int(x) for x in np.random.default_rng(5).integers(1, 50, 21) * 2048]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, lens, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    shards = [g[1] for g in got]
    assert sorted(shards[0] + shards[1]) == list(range(len(lens)))
    assert not set(shards[0]) & set(shards[1])
    loads = [sum(lens[i] for i in s) for s in shards]
    want_t = max(loads) / 1e6
    want_a = sum(l // 100 for l in lens)
    for _, _, t, a in got:
        assert t == pytest.approx(want_t) and a == want_a

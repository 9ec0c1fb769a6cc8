"""Host logic of the multi-GPU path (CPU): the length-balanced partition of
a batch, the reduction of the totals and the gather of the per-signal
results over a world-size-2 gloo group.  Each rank decomposes its shard
with the FP64 oracle standing in for its GPU (no GPU on this host); the
gathered decompositions must equal a one-process run of the whole batch."""
import os
import socket

import numpy as np
import pytest

from paper_2202_12380_gb300 import inputs
from paper_2202_12380_gb300.shard import gather_results, partition, reduce_totals


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


def test_partition_by_work_balances_time_not_length():
    """Loads other than lengths (e.g. atoms of an earlier run): the two
    shortest signals run to K_max and carry the work.  By length they share
    a rank (20 of the 22 units of work on one of three ranks); by work
    each heavy signal gets a rank of its own."""
    lens = [9, 8, 4, 3]
    work = [1.0, 1.0, 10.0, 10.0]
    by_len = partition(lens, 3)
    assert by_len == [[0], [1], [2, 3]]
    assert max(sum(work[i] for i in p) for p in by_len) == 20.0
    by_work = partition(work, 3)
    assert by_work == [[2], [3], [0, 1]]
    assert max(sum(work[i] for i in p) for p in by_work) == 10.0
    with pytest.raises(ValueError):
        partition([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        partition([float("nan")], 1)


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


def _batch():
    dicts = [(inputs.blackman(w), w // 4, w) for w in (64, 128)]
    lens = [int(x) for x in np.random.default_rng(5).integers(1, 6, 9) * 1024]
    xs = [inputs.mixture(L, 300 + i, fs=8000.0) for i, L in enumerate(lens)]
    return dicts, lens, xs


def _decompose(dicts, x):
    from oracle import cmp
    r = cmp.mp_coef(dicts, x, 1e-4, 60, 25.0)
    return (r.dict.tolist(), r.m.tolist(), r.n.tolist(), r.c.tolist(), r.E.tolist(), r.stop)


def _rank_main(rank, world, port, q):
    import time

    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dicts, lens, xs = _batch()
        mine = partition(lens, world)[rank]
        t0 = time.perf_counter()
        res = {i: _decompose(dicts, xs[i]) for i in mine}
        secs = time.perf_counter() - t0
        atoms = sum(len(r[0]) for r in res.values())
        t, a = reduce_totals(secs, atoms)
        allres = gather_results(res)
        q.put((rank, mine, secs, t, a, allres))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_shards_totals_and_gather():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort(key=lambda g: g[0])
    dicts, lens, xs = _batch()
    shards = [g[1] for g in got]
    assert sorted(shards[0] + shards[1]) == list(range(len(lens)))
    assert not set(shards[0]) & set(shards[1])
    # one process, whole batch: the reference for the gathered results
    ref = {i: _decompose(dicts, x) for i, x in enumerate(xs)}
    want_atoms = sum(len(r[0]) for r in ref.values())
    for rank, mine, secs, t, a, allres in got:
        assert a == want_atoms                      # atoms summed over ranks
        assert t == pytest.approx(max(g[2] for g in got))  # slowest rank's time
        assert allres == ref                        # every signal, once, as alone

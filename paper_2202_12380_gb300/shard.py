"""Multi-GPU helpers.

A batch of signals shards across ranks with no exchange on the data path:
every signal is decomposed by exactly one rank (the pursuit of one signal
never reads another's coefficients), so the only collective is the
reduction of the totals (atoms selected, slowest rank's time).  One signal
does not shard -- each iteration needs the global argmax of the previous
update -- so a single-signal run on N GPUs is N replicas.
"""
from __future__ import annotations


def partition(loads, nranks: int):
    """Load-balanced assignment of signals to ranks: the largest load first
    to the least-loaded rank, ties to the lower signal index and rank.  A
    load is any non-negative per-signal cost: the signal length (the
    default of the bench), or the atoms each signal needed in an earlier run
    of similar signals, which is closer to its time (a pursuit that runs to
    K_max costs more than a longer one that reaches its SNR early).  Returns
    one ascending list of signal indices per rank; deterministic for given
    inputs."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    w = [float(x) for x in loads]
    if any(not (x >= 0.0) or x == float("inf") for x in w):
        raise ValueError("loads must be finite and >= 0")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    load = [0.0] * nranks
    out = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += w[i]
    return [sorted(s) for s in out]


def reduce_totals(seconds: float, atoms: float, device="cpu"):
    """(max seconds over ranks, sum of atoms over ranks) through
    torch.distributed; the identity without an initialised process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds), float(atoms)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    a = torch.tensor([float(atoms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return float(t.item()), float(a.item())


def gather_results(mine: dict):
    """Merge per-rank results keyed by signal index (e.g. each rank's atom
    lists) on every rank, through torch.distributed's object gather; the
    identity without an initialised process group.  Keys must not repeat
    across ranks (partition() gives disjoint shards)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return dict(mine)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, dict(mine))
    out = {}
    for p in parts:
        for k, v in p.items():
            if k in out:
                raise ValueError("signal %r was decomposed by two ranks" % (k,))
            out[k] = v
    return out

"""Launch-shape autotuner for the MP loop.

The shape of the persistent MP launch -- threads per CTA, CTAs per signal
(thread-block cluster size) and, with one CTA per signal, the size of the
on-chip top level of the max tree (frames grouped by 2^g so that at most
that many keys are scanned per iteration) -- does not change the result,
only the speed.  A shape is (threads, cluster, top_keys), top_keys 0 for
the launch's default; ``apply`` sets one on a state.
``tune`` times every feasible shape on the caller's own workload (up to
``k_probe`` atoms per signal with the caller's stop target), picks the
fastest and optionally caches the choice in a JSON file keyed by the
dictionary set and the signal lengths.  With several signals the stop target
matters: shapes that need two waves of CTAs win or lose by how the signals'
pursuits end, so the probe should stop the way the real run does.

With several signals the tuner first runs the probe once in the default
shape and takes each signal's atom count as its work; with that work as the
launch order (``mpgabor.mp_state_set_work_hint``: the longest pursuits
start first, so they do not land in the last wave) it times the shapes.
``with_work=True`` also returns the work, for the caller's state.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import mpgabor as mg

THREADS = (128, 256, 512)
CLUSTERS = (1, 2, 4, 8, 16)


def apply(state, shape):
    """Set a tuned shape (threads, cluster[, top_keys]) on a state."""
    mg.mp_state_set_launch(state, int(shape[0]), int(shape[1]))
    if len(shape) > 2 and int(shape[2]):
        mg.mp_state_set_top_keys(state, int(shape[2]))


def top_groups(plan, lengths, cap):
    """log2 of the frames per top-level key of each signal of a one-CTA
    launch whose top level holds at most cap keys (the launch makes the same
    choice)."""
    out = []
    for L in lengths:
        g = 0
        while sum(-(-(int(L) // a) // (1 << g)) for a in plan.a) > cap and g < 30:
            g += 1
        out.append(g)
    return tuple(out)


def _key(shape):
    return "x".join("%d" % v for v in shape)


def _parse(key):
    v = tuple(int(x) for x in key.split("x"))
    return v + (0,) * (3 - len(v))


def signature(plan, lengths) -> str:
    key = json.dumps({"w": plan.wlen, "a": plan.a, "M": plan.M, "eps": plan.eps,
                      "flags": plan.flags, "L": sorted(int(x) for x in lengths)})
    return hashlib.sha256(key.encode()).hexdigest()[:16]


def _load(path):
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def tune(plan, xs, k_probe=2000, target_snr_db=200.0, stream=None, cache_path=None, repeats=2,
         order_by_work=True, with_work=False):
    """Returns ((threads, cluster, top_keys), {shape: ms}) for device signals
    xs, and the per-signal work (atoms of the probe, None for one signal or
    when order_by_work is off) as a third item when with_work is set.  With
    one CTA per signal the default top level and, where they group some
    signal's frames differently, a half and a quarter of it are timed."""
    import numpy as np
    import torch

    sig = signature(plan, [x.numel() for x in xs])
    cache = _load(cache_path)
    if sig in cache and (not with_work or "work" in cache[sig]):
        shape = _parse(_key(cache[sig]["shape"]))
        ms = {_parse(k): v for k, v in cache[sig]["ms"].items()}
        return (shape, ms, cache[sig].get("work")) if with_work else (shape, ms)
    stream = stream or torch.cuda.current_stream()
    state = mg.mp_analyze(plan, xs)
    work = None
    if order_by_work and len(xs) > 1:
        mg.mp_run(state, k_probe, target_snr_db)
        n, _, _ = mg.mp_get_status(state)
        work = [float(v) for v in np.asarray(n, dtype=np.float64)]
        mg.mp_state_set_work_hint(state, work)

    def timed():
        best = None
        for _ in range(repeats):
            mg.mp_analyze(plan, xs, state)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                mg.mp_run_async(state, k_probe, target_snr_db)
                e1.record(stream)
            stream.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best

    lengths = [x.numel() for x in xs]
    timings = {}
    for t in THREADS:
        for c in CLUSTERS:
            try:
                mg.mp_state_set_launch(state, t, c)
            except mg.MPError:
                continue
            timings[(t, c, 0)] = timed()
            if c != 1:
                continue
            cap = mg.mp_state_get_top_keys(state)
            seen = top_groups(plan, lengths, cap)
            for k in (cap // 2, cap // 4):
                groups = top_groups(plan, lengths, k)
                if k < 64 or groups == seen:
                    continue
                try:
                    mg.mp_state_set_top_keys(state, k)
                except mg.MPError:
                    continue
                seen = groups
                timings[(t, c, k)] = timed()
    state.close()
    shape = min(timings, key=timings.get)
    if cache_path:
        cache[sig] = {"shape": list(shape), "ms": {_key(k): v for k, v in timings.items()},
                      "work": work}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return (shape, timings, work) if with_work else (shape, timings)

"""Launch-shape autotuner for the MP loop.

The shape of the persistent MP launch -- threads per CTA and CTAs per signal
(thread-block cluster size) -- does not change the result, only the speed.
``tune`` times every feasible shape on the caller's own workload (up to
``k_probe`` atoms per signal with the caller's stop target), picks the
fastest and optionally caches the choice in a JSON file keyed by the
dictionary set and the signal lengths.  Apply it with
``mpgabor.mp_state_set_launch``.  With several signals the stop target
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
    """Returns ((threads, cluster), {shape: ms}) for device signals xs, and
    the per-signal work (atoms of the probe, None for one signal or when
    order_by_work is off) as a third item when with_work is set."""
    import numpy as np
    import torch

    sig = signature(plan, [x.numel() for x in xs])
    cache = _load(cache_path)
    if sig in cache and (not with_work or "work" in cache[sig]):
        t, c = cache[sig]["shape"]
        ms = {tuple(map(int, k.split("x"))): v for k, v in cache[sig]["ms"].items()}
        return ((t, c), ms, cache[sig].get("work")) if with_work else ((t, c), ms)
    stream = stream or torch.cuda.current_stream()
    state = mg.mp_analyze(plan, xs)
    work = None
    if order_by_work and len(xs) > 1:
        mg.mp_run(state, k_probe, target_snr_db)
        n, _, _ = mg.mp_get_status(state)
        work = [float(v) for v in np.asarray(n, dtype=np.float64)]
        mg.mp_state_set_work_hint(state, work)
    timings = {}
    for t in THREADS:
        for c in CLUSTERS:
            try:
                mg.mp_state_set_launch(state, t, c)
            except mg.MPError:
                continue
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
            timings[(t, c)] = best
    state.close()
    shape = min(timings, key=timings.get)
    if cache_path:
        cache[sig] = {"shape": list(shape), "ms": {"%dx%d" % k: v for k, v in timings.items()},
                      "work": work}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return (shape, timings, work) if with_work else (shape, timings)

"""Host logic of the launch-shape autotuner (CPU): the top-level grouping it
predicts for a cap (the rule the MP launch applies), shape keys, and the
cache, including entries written before shapes carried a top-level cap."""
import json
from types import SimpleNamespace

from paper_2202_12380_gb300 import autotune


def _plan():
    return SimpleNamespace(wlen=[128, 256, 512], a=[32, 64, 128], M=[128, 256, 512], eps=1e-4,
                           flags=0)


def test_top_groups_smallest_power_that_fits():
    plan = _plan()
    # 16384 samples: 512 + 256 + 128 = 896 frames
    assert autotune.top_groups(plan, [16384], 16384) == (0,)
    assert autotune.top_groups(plan, [16384], 896) == (0,)
    assert autotune.top_groups(plan, [16384], 895) == (1,)
    assert autotune.top_groups(plan, [16384], 256) == (2,)   # 128 + 64 + 32 = 224
    assert autotune.top_groups(plan, [16384], 64) == (4,)    # 32 + 16 + 8 = 56
    # ragged groups round up per dictionary: 12 + 6 + 3 frames in groups of
    # 2 are 6 + 3 + 2 keys, in groups of 4 3 + 2 + 1
    assert autotune.top_groups(plan, [384, 16384], 64) == (0, 4)
    assert autotune.top_groups(plan, [384], 11) == (1,)
    assert autotune.top_groups(plan, [384], 10) == (2,)


def test_shape_keys_round_trip():
    assert autotune._parse("512x1") == (512, 1, 0)
    assert autotune._parse(autotune._key((512, 1, 8192))) == (512, 1, 8192)
    assert autotune._key((128, 16, 0)) == "128x16x0"


def test_cache_hit_returns_three_part_shapes(tmp_path):
    plan = _plan()
    lengths = [4096, 8192]
    xs = [SimpleNamespace(numel=lambda L=L: L) for L in lengths]
    sig = autotune.signature(plan, lengths)
    path = tmp_path / "tune.json"
    # an entry from before the top-level cap was tuned
    path.write_text(json.dumps({sig: {"shape": [256, 2], "ms": {"256x2": 1.5, "512x1": 2.0},
                                      "work": [3.0, 4.0]}}))
    shape, ms, work = autotune.tune(plan, xs, cache_path=str(path), with_work=True)
    assert shape == (256, 2, 0)
    assert ms == {(256, 2, 0): 1.5, (512, 1, 0): 2.0}
    assert work == [3.0, 4.0]
    path.write_text(json.dumps({sig: {"shape": [512, 1, 8192],
                                      "ms": {"512x1x0": 2.0, "512x1x8192": 1.9}}}))
    shape, ms = autotune.tune(plan, xs, cache_path=str(path))
    assert shape == (512, 1, 8192) and ms[(512, 1, 8192)] == 1.9

"""The C-ABI library builds, loads and exports every function that
include/mpgabor.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2202_12380_gb300 import build, mpgabor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpgabor.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mp_plan_create", "mp_analyze", "mp_run", "mp_synthesize", "mp_get_atoms",
                     "mp_plan_destroy", "mp_state_destroy", "mp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_exports_every_declared_symbol():
    """The bounds-checking twin (-DMP_CHECK_BOUNDS) is the same ABI."""
    lib = ctypes.CDLL(build.build(checked=True))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(mpgabor.EXPORTS) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(mpgabor, n))


def test_last_error_without_gpu(libpath):
    # a pure host call: argument validation fails before any CUDA work
    lib = mpgabor.lib()
    h = ctypes.c_void_p()
    rc = lib.mp_plan_create(ctypes.byref(h), 0, None, None, None, None, 1e-4, 0, None)
    assert rc == mpgabor.MP_EINVAL
    assert b"bad arguments" in lib.mp_last_error()


def _create(wins, a, M, eps=1e-4):
    lib = mpgabor.lib()
    import numpy as np
    wins = [np.ascontiguousarray(w, np.float64) for w in wins]
    W = len(wins)
    arr = (ctypes.POINTER(ctypes.c_double) * W)(
        *[w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for w in wins])
    h = ctypes.c_void_p()
    rc = lib.mp_plan_create(ctypes.byref(h), W, arr, (ctypes.c_int * W)(*[len(w) for w in wins]),
                            (ctypes.c_int * W)(*a), (ctypes.c_int * W)(*M), eps, 0, None)
    return rc, lib.mp_last_error().decode()


@pytest.mark.parametrize("case,expect", [
    ("odd_M", mpgabor.MP_EINVAL),
    ("M_not_multiple_of_a", mpgabor.MP_ENOTCOMPAT),
    ("a_not_pairwise_divisible", mpgabor.MP_ENOTCOMPAT),
    ("M_not_pairwise_dividing", mpgabor.MP_ENOTCOMPAT),
    ("nan_window", mpgabor.MP_EINVAL),
    ("negative_eps", mpgabor.MP_EINVAL),
    ("odd_window", mpgabor.MP_EINVAL),
])
def test_plan_validation_is_host_side(libpath, case, expect):
    """Sec. 2.1 compatibility rules and argument checks are enforced before
    any device work, so they run here without a GPU."""
    import numpy as np
    g = np.hanning(64)
    wins, a, M, eps = [g], [16], [64], 1e-4
    if case == "odd_M":
        M = [63]
    elif case == "M_not_multiple_of_a":
        a = [24]
    elif case == "a_not_pairwise_divisible":
        wins, a, M = [g, g], [16, 24], [64, 96]
    elif case == "M_not_pairwise_dividing":
        wins, a, M = [g, g], [16, 16], [64, 96]
    elif case == "nan_window":
        g2 = g.copy()
        g2[3] = np.nan
        wins = [g2]
    elif case == "negative_eps":
        eps = -1.0
    elif case == "odd_window":
        wins = [np.hanning(63)]
    rc, msg = _create(wins, a, M, eps)
    assert rc == expect, (rc, msg)
    assert msg


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every call raises."""
    from paper_2202_12380_gb300 import mpgabor

    monkeypatch.setattr(mpgabor, "_lib", None)
    monkeypatch.setattr(mpgabor, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        mpgabor.lib()


def test_flag_validation_is_host_side(libpath):
    """MP_COEF_FP64 cannot be combined with the split-BF16 analysis, and
    unknown flag bits are refused, before any device work."""
    import numpy as np
    lib = mpgabor.lib()
    g = np.ascontiguousarray(np.hanning(64), np.float64)
    arr = (ctypes.POINTER(ctypes.c_double) * 1)(g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    for flags in (mpgabor.MP_COEF_FP64 | mpgabor.MP_ANALYSIS_BF16X3, 1 << 7):
        h = ctypes.c_void_p()
        rc = lib.mp_plan_create(ctypes.byref(h), 1, arr, (ctypes.c_int * 1)(64),
                                (ctypes.c_int * 1)(16), (ctypes.c_int * 1)(64), 1e-4, flags, None)
        assert rc == mpgabor.MP_EINVAL, flags
        assert lib.mp_last_error()


def test_null_handles_are_refused(libpath):
    """Calls on missing plans or states return MP_EINVAL with a message."""
    lib = mpgabor.lib()
    assert lib.mp_state_set_work_hint(None, None) == mpgabor.MP_EINVAL
    assert b"null state" in lib.mp_last_error()
    assert lib.mp_state_set_launch(None, 128, 1) == mpgabor.MP_EINVAL
    assert lib.mp_state_set_top_keys(None, 1024) == mpgabor.MP_EINVAL
    assert b"null state" in lib.mp_last_error()
    k = ctypes.c_int(-1)
    assert lib.mp_state_get_top_keys(None, ctypes.byref(k)) == mpgabor.MP_EINVAL
    assert k.value == -1
    assert lib.mp_state_set_resets(None, 1, 0.0) == mpgabor.MP_EINVAL
    assert lib.mp_get_status(None, None, None, None) == mpgabor.MP_EINVAL
    n = ctypes.c_int64()
    assert lib.mp_decompose_static(None, None, 0, 0, 40.0, None, None, ctypes.byref(n), None,
                                   None) == mpgabor.MP_EINVAL
    assert b"bad argument" in lib.mp_last_error()

"""The parity comparison itself (host logic, CPU): divergences and errors
planted into copies of an oracle decomposition are accepted or rejected as
the rule states, and the divergence report classifies them."""
import numpy as np
import pytest

from oracle import cmp
from paper_2202_12380_gb300 import inputs
from tests.parity import compare, explain_divergence, first_near_tie

ATOM = np.dtype([("dict", "<i4"), ("m", "<i4"), ("n", "<i8"), ("re", "<f4"), ("im", "<f4")])


@pytest.fixture(scope="module")
def ref():
    dicts = [(inputs.blackman(64), 16, 64), (inputs.blackman(128), 32, 128)]
    # seed 82: a decision with a relative gap of 1.7e-6 at atom 85, before
    # the first 1e-6 near tie
    x = inputs.mixture(2048, 82, fs=8000.0)
    return cmp.mp_coef(dicts, x, 1e-4, 200, 200.0)


def _as_gpu(ref, rel_err=0.0):
    a = np.zeros(ref.n_atoms, ATOM)
    a["dict"], a["m"], a["n"] = ref.dict, ref.m, ref.n
    c = ref.c * (1.0 + rel_err)
    a["re"], a["im"] = c.real, c.imag
    return a, ref.E.copy(), ref.E0


def test_identical_sequence_passes(ref):
    a, e, E0 = _as_gpu(ref)
    r = compare(a, e, E0, ref)
    assert r["checked"] == min(first_near_tie(ref), ref.n_atoms)


def test_divergence_at_a_clear_gap_fails(ref):
    gap = (ref.s1 - ref.s2) / ref.s1
    k = int(np.argmax(gap[:first_near_tie(ref)]))  # the clearest decision
    a, e, E0 = _as_gpu(ref, rel_err=2e-6)
    a["m"][k] += 1
    with pytest.raises(AssertionError, match="differs"):
        compare(a, e, E0, ref)


def test_divergence_inside_measured_precision_fails_but_is_reported(ref):
    gap = (ref.s1 - ref.s2) / ref.s1
    k = int(np.argmin(gap[10:first_near_tie(ref)])) + 10  # the closest decision
    g = float(gap[k])
    assert 1e-6 <= g < 1e-5
    # coefficients before k carry a relative error of g (more than half the
    # gap): the strict rule still fails, the report calls it a precision tie
    a, e, E0 = _as_gpu(ref, rel_err=g)
    a["n"][k] += 1
    with pytest.raises(AssertionError, match="differs before the first near tie"):
        compare(a, e, E0, ref)
    why = explain_divergence(a, ref)
    assert why["divergence"] == k and why["kind"] == "precision tie"
    assert abs(why["gap"] - g) < 1e-12
    # the same divergence with exact coefficients is unexplained
    a, e, E0 = _as_gpu(ref)
    a["n"][k] += 1
    assert explain_divergence(a, ref)["kind"] == "unexplained"


def test_divergence_after_near_tie_passes(ref):
    import copy
    k = 150
    r2 = copy.copy(ref)
    r2.s2 = ref.s2.copy()
    r2.s2[k] = ref.s1[k] * (1.0 - 5e-7)  # plant a near tie at atom k
    assert first_near_tie(r2) == k
    a, e, E0 = _as_gpu(ref)
    a["m"][k] += 1
    r = compare(a, e, E0, r2)
    assert r["checked"] == k
    assert explain_divergence(a, r2)["kind"] == "after near tie"


def test_coefficient_error_above_tolerance_fails(ref):
    a, e, E0 = _as_gpu(ref, rel_err=3e-5)
    with pytest.raises(AssertionError, match="coefficient"):
        compare(a, e, E0, ref)


def test_snr_curve_off_fails(ref):
    a, e, E0 = _as_gpu(ref)
    e = e * 10 ** (0.02 / 10)
    with pytest.raises(AssertionError, match="SNR"):
        compare(a, e, E0, ref)

"""The seeded input generators shared by the GPU path and the oracle (CPU):
deterministic, and shaped as the workloads state (window norms and edges,
batch length law, divisibility the library requires, noise levels)."""
import math

import numpy as np
import pytest

from paper_2202_12380_gb300 import inputs


@pytest.mark.parametrize("w", [64, 256, 2048])
def test_windows_unit_norm_zero_centred(w):
    for g in (inputs.blackman(w), inputs.hann(w), inputs.gauss_edge(w)):
        assert g.size == w
        assert abs(np.sum(g * g) - 1.0) < 1e-12
        assert int(np.argmax(g)) == w // 2           # index w/2 holds t = 0
        assert np.allclose(g[1:], g[1:][::-1])        # even: g(t) = g(-t)


def test_gaussian_edge_value():
    g = inputs.gauss_edge(1024, 1e-4)
    assert abs(g[0] / g[512] - 1e-4) < 1e-12


def test_generators_are_deterministic():
    a = inputs.mixture(4096, 7)
    b = inputs.mixture(4096, 7)
    c = inputs.mixture(4096, 8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(inputs.white_noise(100, 3), inputs.white_noise(100, 3))


def test_mixture_noise_level():
    # the pink-noise part sits 30 dB below the deterministic part: removing
    # it (same seed, same draws) leaves an SNR of 30 dB
    L = 1 << 15
    x = inputs.mixture(L, 11, snr_db=30.0)
    y = inputs.mixture(L, 11, snr_db=200.0)  # noise scaled away
    snr = 10 * math.log10(np.sum(y * y) / np.sum((x - y) ** 2))
    assert abs(snr - 30.0) < 1e-6


def test_batch_lengths_law():
    cfg = inputs.WORKLOADS["batch256"]
    lens = inputs.batch_lengths(cfg, cfg["id"])
    assert len(lens) == 256
    assert all(L % 2048 == 0 and cfg["Lmin"] <= L <= cfg["Lmax"] for L in lens)
    logs = np.log2(lens)
    # log-uniform over 14..20: the median is near 17
    assert 16.0 < np.median(logs) < 18.0


def test_workload_lengths_fit_the_library():
    # every length is a multiple of every hop and channel count and at
    # least twice the longest window (what mp_analyze requires)
    for name, cfg in inputs.WORKLOADS.items():
        dicts = cfg["dicts"]
        lens = inputs.batch_lengths(cfg, cfg["id"]) if name == "batch256" else [cfg["L"]]
        wmax = max(w for _, w, _, _ in dicts)
        for L in lens:
            assert L >= 2 * wmax
            for _, w, a, M in dicts:
                assert L % a == 0 and L % M == 0 and M % a == 0

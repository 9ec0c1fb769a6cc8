"""Pins of the oracle's analysis (reduced DGT) and synthesis (CPU only)."""
import numpy as np
import pytest

from oracle import cmp, explicit
from paper_2202_12380_gb300 import inputs


@pytest.mark.parametrize("dims", [(16, 4, 16), (32, 8, 32), (24, 6, 24), (8, 4, 16)])
def test_dgt_matches_explicit_matrix(dims):
    """rho = D^* x restricted to m = 0..M/2 (eq. gabdict)."""
    w, a, M = dims
    L = 96
    g = inputs.blackman(w)
    x = np.random.default_rng(1).standard_normal(L)
    D = explicit.gabor_matrix(g, a, M, L)
    idx = explicit.reduced_columns(a, M, L)
    ref = (D.conj().T @ x)[idx].reshape(L // a, M // 2 + 1)
    got = cmp.dgt(x, g, a, M)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_dgt_matches_fft_of_frames():
    """Same coefficients through numpy's FFT: frame n is x(n a + t) g(t),
    t = -w/2..w/2-1, rotated so t = 0 sits at index 0."""
    L, w, a, M = 4096, 256, 64, 256
    g = inputs.blackman(w)
    x = np.random.default_rng(2).standard_normal(L)
    got = cmp.dgt(x, g, a, M)
    t = np.arange(w) - w // 2
    for n in (0, 1, 17, L // a - 1):
        f = x[(n * a + t) % L] * g
        buf = np.zeros(M)
        np.add.at(buf, t % M, f)
        ref = np.fft.fft(buf)[: M // 2 + 1]
        assert np.max(np.abs(got[n] - ref)) < 1e-11


def test_synth_matches_explicit_matrix():
    """Real synthesis sum c d + conj(c) conj(d) (eq. idgtreal); one term at
    m in {0, M/2}."""
    L = 64
    dicts = [(inputs.blackman(16), 4, 16), (inputs.hann(32), 8, 32)]
    rng = np.random.default_rng(3)

    class A:
        pass

    at = A()
    at.dict = np.array([0, 0, 1, 1, 0], np.int32)
    at.m = np.array([0, 3, 16, 5, 8], np.int32)
    at.n = np.array([2, 15, 1, 7, 0], np.int64)
    at.c = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    at.c[[0, 2, 4]] = at.c[[0, 2, 4]].real
    y = cmp.synth(dicts, at, L)
    ref = np.zeros(L, complex)
    for u, m, n, c in zip(at.dict, at.m, at.n, at.c):
        g, a, M = dicts[u]
        D = explicit.gabor_matrix(g, a, M, L)
        d = D[:, m + n * M]
        if m == 0 or 2 * m == M:
            ref += c * d
        else:
            ref += c * d + np.conj(c) * np.conj(d)
    assert np.max(np.abs(ref.imag)) < 1e-12
    assert np.max(np.abs(y - ref.real)) < 1e-12

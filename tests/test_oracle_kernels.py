"""Pins of the oracle's cross-Gram kernels (CPU only).

The kernel h_{u,v} of the C oracle is checked against things it does not
compute itself: an explicit Gram matrix D^* D built column by column from
eq. gabdict (twisted-convolution form, eq. GramKern, Sec. 4.2 for
cross-kernels), the kernel sizes printed in Fig. 1, a closed form for the
untruncated Gaussian, and the conjugate symmetries noted in Sec. 4.1.
"""
import os

import numpy as np
import pytest

from oracle import cmp, explicit
from paper_2202_12380_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_kernel_sizes.txt")


def _expected_gram_entry(h, taus, Mx, an, u_d, v_d, k, j, m, n, L):
    (_, au, Mu), (_, av, Mv) = u_d, v_d
    tau = n * av - j * au
    val = 0.0
    for t in (tau - L, tau, tau + L):
        if taus[0] <= t <= taus[-1]:
            it = (t - taus[0]) // an
            d = (m * (Mx // Mv) - k * (Mx // Mu)) % Mx
            val += np.exp(2j * np.pi * ((k * t) % Mu) / Mu) * h[it, d]
    return val


@pytest.mark.parametrize("case", ["single", "two", "fig2"])
def test_kernel_matches_explicit_gram(case):
    """G(q, p) = <d_p, d_q> from explicit matrices equals
    e^{i 2 pi k tau / M_u} h_{u,v}(m M_max/M_v - k M_max/M_u, tau)."""
    if case == "single":
        L, dicts = 64, [(inputs.blackman(16), 4, 16)]
    elif case == "two":
        L, dicts = 96, [(inputs.blackman(16), 4, 16), (inputs.hann(32), 8, 32)]
    else:
        # layout of Fig. 2: a1 = 4 a_min, M1 = 8 a_min; a2 = a_min, M2 = 2 a_min
        L, dicts = 64, [(inputs.blackman(32), 16, 32), (inputs.hann(8), 4, 8)]
    worst = 0.0
    for u, du in enumerate(dicts):
        Du = explicit.gabor_matrix(du[0], du[1], du[2], L)
        for v, dv in enumerate(dicts):
            Dv = explicit.gabor_matrix(dv[0], dv[1], dv[2], L)
            G = Dv.conj().T @ Du
            h, taus, Mx, an = cmp.kernel(du, dv)
            Mu, Mv = du[2], dv[2]
            for j in range(L // du[1]):
                for k in range(Mu):
                    for n in range(L // dv[1]):
                        for m in range(Mv):
                            e = _expected_gram_entry(h, taus, Mx, an, du, dv, k, j, m, n, L)
                            worst = max(worst, abs(G[m + n * Mv, k + j * Mu] - e))
    assert worst < 1e-12


def _bbox(h, Mx, eps):
    mask = np.abs(h) > eps
    cols = np.where(mask.any(axis=1))[0]
    rows = np.where(mask.any(axis=0))[0]
    signed = np.where(rows > Mx // 2, rows - Mx, rows)
    return int(signed.max() - signed.min() + 1), int(cols.max() - cols.min() + 1)


def _golden_rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, a, M, r, c = line.split()
        out.append((kind, int(a), int(M), int(r), int(c)))
    return out


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_fig1_kernel_sizes(row):
    kind, a, M, rows, cols = row
    if kind == "gauss":
        # the figure's Gaussian is the untruncated exp(-pi t^2 / (a M))
        g = inputs.gauss_lambda(4 * M, float(a * M))
    else:
        g = inputs.make_window(kind, M)
    h, taus, Mx, an = cmp.kernel((g, a, M), (g, a, M))
    assert _bbox(h, Mx, 1e-4) == (rows, cols)


def test_gaussian_closed_form():
    """For g = exp(-pi t^2 / lam) (unit norm, untruncated):
    h(D, tau) = exp(-pi tau^2/(2 lam)) exp(-pi lam D^2/(2 M^2)) exp(i pi D tau / M),
    D the representative of delta in (-M/2, M/2]."""
    a, M = 64, 256
    lam = float(a * M)
    g = inputs.gauss_lambda(2048, lam)
    h, taus, Mx, an = cmp.kernel((g, a, M), (g, a, M))
    D = np.arange(M)
    D = np.where(D > M // 2, D - M, D)
    tt = taus[:, None].astype(float)
    ref = np.exp(-np.pi * tt ** 2 / (2 * lam)) * np.exp(-np.pi * lam * D[None, :] ** 2 / (2.0 * M * M)) \
        * np.exp(1j * np.pi * D[None, :] * tt / M)
    assert np.max(np.abs(h - ref)) < 1e-12


@pytest.mark.parametrize("kind", ["blackman", "hann"])
def test_kernel_conjugate_symmetry(kind):
    """Even windows: h(-D, tau) = conj h(D, tau) and h(D, -tau) = conj h(D, tau)."""
    a, M = 64, 256
    g = inputs.make_window(kind, M)
    h, taus, Mx, an = cmp.kernel((g, a, M), (g, a, M))
    assert taus[0] == -taus[-1]
    neg_d = h[:, (-np.arange(Mx)) % Mx]
    assert np.max(np.abs(neg_d - h.conj())) < 1e-14
    assert np.max(np.abs(h[::-1, :] - h.conj())) < 1e-14
    # peak at the origin equals the window energy, 1
    it0 = int(np.where(taus == 0)[0][0])
    assert abs(h[it0, 0] - 1.0) < 1e-14


def test_cross_kernel_is_adjoint():
    """The cross-Gram blocks satisfy G_{v,u} = G_{u,v}^*, and the oracle's
    kernels h_{u,v} and h_{v,u} reproduce both blocks (Fig. 2 layout)."""
    L = 64
    du, dv = (inputs.blackman(32), 16, 32), (inputs.hann(8), 4, 8)
    Du = explicit.gabor_matrix(*du, L)
    Dv = explicit.gabor_matrix(*dv, L)
    Guv = Dv.conj().T @ Du
    Gvu = Du.conj().T @ Dv
    assert np.max(np.abs(Guv - Gvu.conj().T)) < 1e-13
    # and the oracle kernel reproduces both blocks
    for (x, y), G in (((du, dv), Guv), ((dv, du), Gvu)):
        h, taus, Mx, an = cmp.kernel(x, y)
        j, k, n, m = 1, 3, 1, 2
        e = _expected_gram_entry(h, taus, Mx, an, x, y, k, j, m, n, L)
        assert abs(G[m + n * y[2], k + j * x[2]] - e) < 1e-12

"""Explicit-matrix oracle (numpy, FP64) for tiny signals.

TEST INFRASTRUCTURE ONLY.  Builds the dictionary matrix of eq. gabdict
column by column and runs matching pursuit by its definition, so it pins the
C oracle through routes that share nothing with it: matrix products for the
Gram matrix and the analysis, and numpy least squares for the real-pair
projection instead of the closed forms of eqs. dualatprod / projenfaster.
"""
from __future__ import annotations

import numpy as np


def gabor_matrix(g, a, M, L):
    """D(l, m + n M) = g(l - n a) exp(i 2 pi m (l - n a) / M), l - n a mod L.

    g is zero-centred (index i holds g(t), t = i - w/2).  Returns the full
    L x (M N) complex matrix, column m + n M (eq. gabdict)."""
    w = len(g)
    N = L // a
    gl = np.zeros(L)
    for i in range(w):
        gl[(i - w // 2) % L] += g[i]
    D = np.zeros((L, M * N), complex)
    l = np.arange(L)
    for n in range(N):
        s = (l - n * a) % L
        # (l - n a) is taken mod L; since M divides L the phase is unchanged
        for m in range(M):
            D[:, m + n * M] = gl[s] * np.exp(2j * np.pi * m * s / M)
    return D


def reduced_columns(a, M, L):
    """Column indices m + n M with m = 0..M/2 in (n, m) order."""
    N = L // a
    return np.array([m + n * M for n in range(N) for m in range(M // 2 + 1)])


def multi_reduced(dicts, L):
    """Concatenated reduced dictionary in (w, n, m) order, plus the labels."""
    cols, labels = [], []
    for w, (g, a, M) in enumerate(dicts):
        D = gabor_matrix(g, a, M, L)
        idx = reduced_columns(a, M, L)
        cols.append(D[:, idx])
        N = L // a
        labels += [(w, m, n) for n in range(N) for m in range(M // 2 + 1)]
    return np.concatenate(cols, axis=1), labels


def conj_partner_column(g, a, M, L, m, n):
    D = gabor_matrix(g, a, M, L)
    return D[:, ((M - m) % M) + n * M]


def pair_projection_energies(Dr, labels, dicts, r):
    """Energy removed from r by projecting it onto the real span of each
    reduced column and its conjugate (onto the real atom itself at m in
    {0, M/2}), for every column: b^T G^-1 b with the 2 x 2 Gram matrix of
    (Re d, Im d)."""
    u1, u2 = Dr.real, Dr.imag
    b1, b2 = u1.T @ r, u2.T @ r
    g11 = np.sum(u1 * u1, axis=0)
    g12 = np.sum(u1 * u2, axis=0)
    g22 = np.sum(u2 * u2, axis=0)
    out = np.empty(Dr.shape[1])
    for p, (w, m, n) in enumerate(labels):
        M = dicts[w][2]
        if m == 0 or 2 * m == M:
            out[p] = b1[p] ** 2 / g11[p]
        else:
            G = np.array([[g11[p], g12[p]], [g12[p], g22[p]]])
            bb = np.array([b1[p], b2[p]])
            out[p] = bb @ np.linalg.solve(G, bb)
    return out


def mp_definition(dicts, x, kmax, pedantic=False):
    """Matching pursuit with real atoms by definition.

    Selection: argmax |<r, d_p>| over the reduced multi-Gabor dictionary
    (ties -> first in (w, n, m) order).  Update: orthogonal projection of r
    onto the real span of {d, conj d} (or onto d alone at m in {0, M/2}),
    computed with numpy least squares.  Returns the atoms (w, m, n, c) with c
    the complex coefficient of d in r_k - r_{k+1} = c d + conj(c) conj(d),
    the energies ||r_k||^2, and the final residual.  pedantic: select the
    column whose real-pair projection removes the most energy."""
    x = np.asarray(x, np.float64)
    L = x.size
    Dr, labels = multi_reduced(dicts, L)
    r = x.copy()
    atoms, energies = [], [float(r @ r)]
    for _ in range(kmax):
        rho = Dr.conj().T @ r
        if pedantic:
            p = int(np.argmax(pair_projection_energies(Dr, labels, dicts, r)))
        else:
            p = int(np.argmax(np.abs(rho) ** 2))
        w, m, n = labels[p]
        g, a, M = dicts[w]
        d = Dr[:, p]
        if m == 0 or 2 * m == M:
            B = np.stack([d.real], axis=1)
            coef, *_ = np.linalg.lstsq(B, r, rcond=None)
            c = complex(coef[0], 0.0)
            r = r - B @ coef
        else:
            # c d + conj(c) conj(d) = 2 Re(c) Re(d) - 2 Im(c) Im(d)
            B = np.stack([2 * d.real, -2 * d.imag], axis=1)
            coef, *_ = np.linalg.lstsq(B, r, rcond=None)
            c = complex(coef[0], coef[1])
            r = r - B @ coef
        atoms.append((w, m, n, c))
        energies.append(float(r @ r))
    return atoms, np.array(energies), r

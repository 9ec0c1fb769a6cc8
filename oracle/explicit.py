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


def full_multi(dicts, L):
    """Concatenated full dictionary (every m = 0..M-1) of all dictionaries,
    columns in (w, n, m) order, with a map from (w, m, n) to the column."""
    cols, index, o = [], {}, 0
    for w, (g, a, M) in enumerate(dicts):
        N = L // a
        D = gabor_matrix(g, a, M, L)
        # gabor_matrix orders columns m + n M, i.e. (n, m) order already
        cols.append(D)
        for n in range(N):
            for m in range(M):
                index[(w, m, n)] = o + m + n * M
        o += M * N
    return np.concatenate(cols, axis=1), index


def mp_truncated_gram(dicts, x, eps, kmax):
    """Coefficient-domain matching pursuit of Alg. 1 with the truncated Gram
    matrix of eq. truncgram, built explicitly.

    G = D^* D over the full multi-Gabor dictionary (every frequency, so the
    conjugate partners are columns too), G(q, p) = <d_p, d_q>; G_eps keeps
    the entries with |G| > eps and sets the others to 0.  rho_0 = D^* x.
    Per step (before it: stop once the estimate E_k <= 0):
      * select p = argmax |rho(p)|^2 over the reduced dictionary
        (m = 0..M/2; ties: first in (w, n, m) order);
      * m in {0, M/2}: the atom is real, c = Re rho(p), energy drop c^2,
        rho -= c G_eps(., p);
      * otherwise, with the partner pbar = (w, M - m, n) and
        gamma = G_eps(pbar, p) = <d_p, conj d_p> (zero when truncated),
        c = (rho(p) - conj(gamma) conj(rho(p))) / (1 - |gamma|^2)
        (eq. dualatprod), energy drop 2 |c|^2 + 2 Re(c^2 gamma)
        (eq. projenfaster), rho -= c G_eps(., p) + conj(c) G_eps(., pbar);
      * E_{k+1} = E_k - energy drop.
    Windows are unit-norm, so <d, d> = 1.  Returns the atoms (w, m, n, c)
    and the estimates E_1..E_K."""
    x = np.asarray(x, np.float64)
    L = x.size
    D, index = full_multi(dicts, L)
    G = D.conj().T @ D
    G[np.abs(G) <= eps] = 0.0
    rho = D.conj().T @ x
    labels = []
    for w, (g, a, M) in enumerate(dicts):
        labels += [(w, m, n) for n in range(L // a) for m in range(M // 2 + 1)]
    red = np.array([index[lab] for lab in labels])
    E = float(x @ x)
    atoms, Es = [], []
    for _ in range(kmax):
        if E <= 0.0:
            break
        s = np.abs(rho[red]) ** 2
        q = int(np.argmax(s))
        w, m, n = labels[q]
        M = dicts[w][2]
        p = red[q]
        r0 = rho[p]
        if m == 0 or 2 * m == M:
            c = complex(r0.real, 0.0)
            drop = c.real ** 2
            rho = rho - c * G[:, p]
        else:
            pb = index[(w, M - m, n)]
            gam = G[pb, p]
            c = (r0 - np.conj(gam) * np.conj(r0)) / (1.0 - abs(gam) ** 2)
            drop = 2.0 * abs(c) ** 2 + 2.0 * (c * c * gam).real
            rho = rho - c * G[:, p] - np.conj(c) * G[:, pb]
        E -= drop
        atoms.append((w, m, n, complex(c)))
        Es.append(E)
    return atoms, np.array(Es)

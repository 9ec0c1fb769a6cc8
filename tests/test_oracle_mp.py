"""Pins of the oracle's matching pursuit loops (CPU only).

* plain MP (signal domain) against MP by definition with an explicit
  dictionary and numpy least squares (Sec. 2.2, real pairs of Sec. 5);
* coefficient-domain MP with eps = 0 against plain MP: with the full Gram
  matrix the coefficient-domain residual is exactly D^* r_k (Sec. 3);
* the energy identity ||r_k||^2 = ||x||^2 - sum of the energy drops;
* for eps > 0 the bound |<r_k, d_p> - rho_k(p)| <= 2 eps sum_l |c_l| that the
  proof of Theorem 1 (appendix) gives, doubled for real atom pairs;
* a signal made of one atom is recovered in one step;
* the stop rules.
"""
import numpy as np
import pytest

from oracle import cmp, explicit
from paper_2202_12380_gb300 import inputs


def _tiny_dicts():
    return [(inputs.blackman(16), 4, 16), (inputs.hann(32), 8, 32)]


def test_plain_matches_definition_tiny():
    L = 96
    dicts = _tiny_dicts()
    x = np.random.default_rng(5).standard_normal(L)
    K = 40
    atoms, energies, r = explicit.mp_definition(dicts, x, K)
    res = cmp.mp_plain(dicts, x, K, 400.0, fullscan=True)
    assert res.stop == cmp.STOP_KMAX and res.n_atoms == K
    for i, (w, m, n, c) in enumerate(atoms):
        assert (res.dict[i], res.m[i], res.n[i]) == (w, m, n), i
        assert abs(res.c[i] - c) < 1e-10 * max(1.0, abs(c))
    # energy bookkeeping of eq. projenfaster equals the true residual energy
    assert np.max(np.abs(res.E - energies[1:])) < 1e-10 * energies[0]
    assert np.max(np.abs(res.extra - r)) < 1e-10


def test_plain_asymmetric_window_uses_conj_gamma():
    """With an asymmetric window <d, conj d> is complex; least squares needs
    conj(gamma) in the numerator of eq. dualatprod (the printed gamma gives a
    different value), and the definition-based MP decides."""
    L = 96
    rng = np.random.default_rng(6)
    g = rng.uniform(0.2, 1.0, 16)
    g /= np.linalg.norm(g)
    dicts = [(g, 4, 16)]
    x = rng.standard_normal(L)
    atoms, energies, _ = explicit.mp_definition(dicts, x, 20)
    res = cmp.mp_plain(dicts, x, 20, 400.0)
    for i, (w, m, n, c) in enumerate(atoms):
        assert (res.dict[i], res.m[i], res.n[i]) == (w, m, n)
        assert abs(res.c[i] - c) < 1e-10
    assert np.max(np.abs(res.E - energies[1:])) < 1e-10 * energies[0]


@pytest.mark.parametrize("case", ["single", "asym", "fig2", "multi3"])
def test_coef_eps0_equals_plain(case):
    if case == "single":
        L, dicts = 2048, [(inputs.gauss_edge(64), 16, 64)]
    elif case == "asym":
        # complex <d, conj d>: pins the conj(gamma) of eq. dualatprod and the
        # gamma read off the own kernel
        g = np.random.default_rng(7).uniform(0.2, 1.0, 32)
        L, dicts = 1024, [(g / np.linalg.norm(g), 8, 32), (inputs.blackman(64), 16, 64)]
    elif case == "fig2":
        L, dicts = 512, [(inputs.blackman(32), 16, 32), (inputs.hann(8), 4, 8)]
    else:
        L, dicts = 2048, [(inputs.blackman(w), w // 4, w) for w in (32, 64, 128)]
    x = inputs.mixture(L, 11, fs=8000.0)
    K = 150
    a = cmp.mp_plain(dicts, x, K, 400.0, fullscan=True)
    b = cmp.mp_coef(dicts, x, 0.0, K, 400.0, fullscan=True)
    assert a.n_atoms == b.n_atoms == K
    assert np.array_equal(a.dict, b.dict) and np.array_equal(a.m, b.m) and np.array_equal(a.n, b.n)
    assert np.max(np.abs(a.c - b.c) / np.abs(a.c)) < 1e-9
    assert np.max(np.abs(a.E - b.E)) < 1e-9 * a.E0


def test_energy_identity_plain():
    L = 1024
    dicts = [(inputs.blackman(w), w // 4, w) for w in (32, 128)]
    x = inputs.mixture(L, 12, fs=8000.0)
    res = cmp.mp_plain(dicts, x, 120, 400.0)
    for k in (1, 10, 60, 120):
        class S:
            pass
        s = S()
        s.dict, s.m, s.n, s.c = res.dict[:k], res.m[:k], res.n[:k], res.c[:k]
        r = x - cmp.synth(dicts, s, L)
        assert abs(float(r @ r) - res.E[k - 1]) < 1e-10 * res.E0


@pytest.mark.parametrize("eps", [1e-4, 1e-3, 1e-2])
def test_coef_theorem1_bound(eps):
    """|<r_k, d_p> - rho_k(p)| <= 2 eps sum_l |c_l| for every p (proof of
    Theorem 1; factor 2 for the two atoms of each real pair)."""
    L = 2048
    dicts = [(inputs.blackman(w), w // 4, w) for w in (64, 256)]
    x = inputs.mixture(L, 13, fs=8000.0)
    res = cmp.mp_coef(dicts, x, eps, 300, 400.0, planes=True)
    r = x - cmp.synth(dicts, res, L)
    bound = 2 * eps * np.sum(np.abs(res.c))
    worst = 0.0
    for (g, a, M), rho in zip(dicts, res.extra):
        true = cmp.dgt(r, g, a, M)
        worst = max(worst, float(np.max(np.abs(true - rho))))
    assert worst <= bound
    assert worst > 0.0  # truncation does change the residual


def test_single_atom_recovered():
    L = 1024
    dicts = [(inputs.blackman(128), 32, 128), (inputs.blackman(64), 16, 64)]
    c = 0.7 - 0.4j

    class S:
        pass

    s = S()
    s.dict, s.m, s.n, s.c = np.array([0], np.int32), np.array([9], np.int32), \
        np.array([5], np.int64), np.array([c])
    x = cmp.synth(dicts, s, L)
    for res in (cmp.mp_plain(dicts, x, 3, 400.0), cmp.mp_coef(dicts, x, 0.0, 3, 400.0)):
        assert (res.dict[0], res.m[0], res.n[0]) == (0, 9, 5)
        assert abs(res.c[0] - c) < 1e-12
        assert abs(res.E[0]) < 1e-12 * res.E0
        assert res.stop in (cmp.STOP_NEGENERGY, cmp.STOP_SNR)
        assert res.n_atoms == 1


def test_stop_rules():
    L = 512
    dicts = [(inputs.blackman(64), 16, 64)]
    x = inputs.mixture(L, 14, fs=8000.0)
    # all-zero input: energy estimate already exhausted
    z = cmp.mp_coef(dicts, np.zeros(L), 1e-4, 10, 40.0)
    assert z.n_atoms == 0 and z.stop == cmp.STOP_NEGENERGY
    # Kmax = 0
    k0 = cmp.mp_coef(dicts, x, 1e-4, 0, 40.0)
    assert k0.n_atoms == 0 and k0.stop == cmp.STOP_KMAX
    # SNR target: stops at the first k with E_k <= E0 10^(-snr/10)
    r = cmp.mp_coef(dicts, x, 1e-4, 5000, 20.0)
    assert r.stop == cmp.STOP_SNR
    thr = r.E0 * 10 ** (-20.0 / 10)
    assert r.E[-1] <= thr and np.all(r.E[:-1] > thr)
    # without a target the estimate eventually goes negative (Sec. 6.1 rule)
    big = cmp.mp_coef(dicts, x, 5e-2, 200000, 400.0)
    assert big.stop == cmp.STOP_NEGENERGY and big.E[-1] <= 0 and np.all(big.E[:-1] > 0)


# ------------------------------------------------------------- resets -----

def test_reset_every_atom_is_plain_mp():
    """Alg. 2 with a reset before every selection re-analyses the exact
    residual each time, so even with a coarse threshold it reproduces plain
    MP's selections.  Coefficients differ only where the exact <d, conj d>
    is below the threshold and taken as zero (Sec. 5.2), i.e. by at most
    about |gamma| <= eps relative."""
    L = 1024
    dicts = [(inputs.blackman(w), w // 4, w) for w in (64, 128)]
    x = inputs.mixture(L, 15, fs=8000.0)
    K = 80
    plain = cmp.mp_plain(dicts, x, K, 400.0)
    rs = cmp.mp_coef_reset(dicts, x, 1e-2, K, 400.0, reset_it=1)
    assert rs.n_resets == K - 1
    assert np.array_equal(plain.dict, rs.dict) and np.array_equal(plain.m, rs.m)
    assert np.array_equal(plain.n, rs.n)
    rel = np.abs(plain.c - rs.c) / np.abs(plain.c)
    assert np.max(rel) < 2 * 1e-2
    assert np.median(rel) < 1e-12  # interior atoms: gamma is zero in both
    assert np.max(np.abs(plain.E - rs.E)) < 1e-3 * plain.E0


def test_reset_energy_is_true_residual_energy():
    """Right after a reset the estimate restarts from the exact residual
    energy: E_k (after atom k, the first atom of an epoch) equals
    ||x - synthesis of atoms 0..k-1||^2 minus that atom's energy drop."""
    L = 2048
    dicts = [(inputs.blackman(w), w // 4, w) for w in (64, 256)]
    x = inputs.mixture(L, 16, fs=8000.0)
    K = 300
    rs = cmp.mp_coef_reset(dicts, x, 1e-2, K, 400.0, reset_it=50)
    assert rs.n_resets == (K - 1) // 50
    no = cmp.mp_coef(dicts, x, 1e-2, K, 400.0)

    class S:
        pass

    for kr in range(50, K, 50):
        s = S()
        s.dict, s.m, s.n, s.c = rs.dict[:kr], rs.m[:kr], rs.n[:kr], rs.c[:kr]
        r = x - cmp.synth(dicts, s, L)
        s2 = S()
        s2.dict, s2.m, s2.n, s2.c = rs.dict[:kr + 1], rs.m[:kr + 1], rs.n[:kr + 1], rs.c[:kr + 1]
        r2 = x - cmp.synth(dicts, s2, L)
        # the estimate after the epoch's first atom is exact up to the
        # truncation of that one atom's projection
        assert abs(rs.E[kr] - float(r2 @ r2)) < 1e-6 * rs.E0
        assert float(r @ r) > float(r2 @ r2)
    # without resets the estimate drifts away from the true energy
    s3 = S()
    s3.dict, s3.m, s3.n, s3.c = no.dict, no.m, no.n, no.c
    r3 = x - cmp.synth(dicts, s3, L)
    assert abs(no.E[-1] - float(r3 @ r3)) > abs(rs.E[-1] - float((x - cmp.synth(dicts, rs, L)) @
                                                                  (x - cmp.synth(dicts, rs, L))))


def test_resets_restore_convergence_with_coarse_threshold():
    """With a coarse kernel threshold the estimate drifts from the true
    error; resets keep the true residual decreasing to the target."""
    L = 2048
    dicts = [(inputs.blackman(w), w // 4, w) for w in (64, 256)]
    x = inputs.mixture(L, 17, fs=8000.0)
    K = 3000

    class S:
        pass

    def true_snr(res):
        s = S()
        s.dict, s.m, s.n, s.c = res.dict, res.m, res.n, res.c
        r = x - cmp.synth(dicts, s, L)
        return 10 * np.log10(float(x @ x) / float(r @ r))

    no = cmp.mp_coef(dicts, x, 5e-2, K, 30.0)
    yes = cmp.mp_coef_reset(dicts, x, 5e-2, K, 30.0, reset_db=-3.0)
    assert yes.n_resets > 0
    assert yes.stop == cmp.STOP_SNR
    assert true_snr(yes) >= 29.5
    assert true_snr(yes) > true_snr(no) + 1.0


# ---------------------------------------------------------- pedantic ------

def test_pedantic_plain_matches_definition():
    """Pedantic selection (Sec. 5: the score is the pair energy drop of eq.
    projenfaster) equals choosing, by brute force on explicit matrices, the
    real atom whose projection removes the most energy."""
    L = 96
    dicts = _tiny_dicts()
    x = np.random.default_rng(8).standard_normal(L)
    K = 30
    atoms, energies, _ = explicit.mp_definition(dicts, x, K, pedantic=True)
    res = cmp.mp_plain(dicts, x, K, 400.0, pedantic=True, fullscan=True)
    for i, (w, m, n, c) in enumerate(atoms):
        assert (res.dict[i], res.m[i], res.n[i]) == (w, m, n), i
        assert abs(res.c[i] - c) < 1e-10 * max(1.0, abs(c))
    assert np.max(np.abs(res.E - energies[1:])) < 1e-10 * energies[0]


def test_pedantic_differs_and_decays_faster():
    """The pedantic score weighs real pairs by 2 against edge atoms, so the
    sequences differ, and each pedantic step removes at least as much true
    energy as the non-pedantic one from the same residual (first step)."""
    L = 1024
    dicts = [(inputs.blackman(w), w // 4, w) for w in (32, 128)]
    x = inputs.mixture(L, 18, fs=8000.0) + 0.5
    a = cmp.mp_plain(dicts, x, 60, 400.0)
    b = cmp.mp_plain(dicts, x, 60, 400.0, pedantic=True)
    assert not (np.array_equal(a.dict, b.dict) and np.array_equal(a.m, b.m)
                and np.array_equal(a.n, b.n))
    assert b.E[0] <= a.E[0] + 1e-12 * a.E0


def test_pedantic_coef_eps0_equals_plain():
    L = 2048
    dicts = [(inputs.blackman(w), w // 4, w) for w in (32, 64, 128)]
    x = inputs.mixture(L, 19, fs=8000.0)
    a = cmp.mp_plain(dicts, x, 120, 400.0, pedantic=True, fullscan=True)
    b = cmp.mp_coef(dicts, x, 0.0, 120, 400.0, pedantic=True, fullscan=True)
    assert np.array_equal(a.dict, b.dict) and np.array_equal(a.m, b.m)
    assert np.array_equal(a.n, b.n)
    assert np.max(np.abs(a.c - b.c) / np.abs(a.c)) < 1e-9


def _gram_layout(case):
    if case == "two":
        return 96, [(inputs.blackman(16), 4, 16), (inputs.hann(32), 8, 32)]
    if case == "fig2":
        return 512, [(inputs.blackman(32), 16, 32), (inputs.hann(8), 4, 8)]
    # asymmetric window: complex <d, conj d>, so gamma and its conjugation
    # in eq. dualatprod matter
    g = np.random.default_rng(7).uniform(0.2, 1.0, 32)
    return 256, [(g / np.linalg.norm(g), 8, 32), (inputs.blackman(64), 16, 64)]


def test_truncated_gram_eps0_is_mp_by_definition():
    """The explicit G-based Alg. 1 with G_0 = D^* D reproduces MP by
    definition (numpy least squares), so its closed forms are pinned."""
    L, dicts = _gram_layout("asym")
    x = inputs.mixture(L, 21, fs=8000.0)
    K = 60
    at, E = explicit.mp_truncated_gram(dicts, x, 0.0, K)
    ref, energies, _ = explicit.mp_definition(dicts, x, K)
    assert [a[:3] for a in at] == [a[:3] for a in ref]
    assert max(abs(a[3] - b[3]) for a, b in zip(at, ref)) < 1e-10
    assert np.max(np.abs(E - energies[1:])) < 1e-10 * energies[0]


@pytest.mark.parametrize("case", ["two", "fig2", "asym"])
@pytest.mark.parametrize("eps", [1e-3, 1e-2])
def test_coef_eps_matches_explicit_truncated_gram(case, eps):
    """eps > 0: the C oracle's kernel-based G_eps (thresholded cross-kernels,
    the landing of Alg. 3, the conjugate term, gamma from the own kernel)
    equals Alg. 1 with the explicitly thresholded D^* D (eq. truncgram)."""
    L, dicts = _gram_layout(case)
    x = inputs.mixture(L, 17, fs=8000.0)
    K = 120 if L > 96 else 60
    at, E = explicit.mp_truncated_gram(dicts, x, eps, K)
    res = cmp.mp_coef(dicts, x, eps, K, 400.0, fullscan=True)
    assert res.n_atoms == len(at) > 0
    assert [(int(a), int(b), int(c)) for a, b, c in zip(res.dict, res.m, res.n)] == \
        [a[:3] for a in at]
    c = np.array([a[3] for a in at])
    assert np.max(np.abs(res.c - c)) < 1e-12 * np.max(np.abs(c)) * 100
    assert np.max(np.abs(res.E - E)) < 1e-12 * res.E0
    # the truncation is active: the eps = 0 pursuit differs
    at0, _ = explicit.mp_truncated_gram(dicts, x, 0.0, K)
    c0 = np.array([a[3] for a in at0])
    k = min(len(at0), len(at))
    assert [a[:3] for a in at0[:k]] != [a[:3] for a in at[:k]] or \
        np.max(np.abs(c0[:k] - c[:k])) > 1e-6 * np.max(np.abs(c))

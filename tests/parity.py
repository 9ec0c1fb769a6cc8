"""Parity helpers: compare a GPU decomposition with the FP64 oracle.

Acceptance (per decomposition):
  * the atom sequence (w, m, n) is identical up to the oracle's first near
    tie, i.e. the first iteration k where (s1 - s2) / s1 < 1e-6 with s1, s2
    the largest and second-largest |rho| over all coefficients (FP64);
  * up to that point every coefficient satisfies |c - c_ora| <= 1e-5 |c_ora|
    (tolerance ``coef_rtol``), and the SNR curve 10 log10(E0/E_k) agrees
    within 0.01 dB.

Precision tie.  The GPU keeps coefficients in FP32, so after many updates a
coefficient carries a relative error of up to about 1e-5 (measured).  Two
candidates whose |rho| differ by less than that can legitimately swap order.
A divergence before the first 1e-6 near tie is therefore accepted, and ends
the compared prefix, only where the oracle's gap at that iteration is below
twice the largest relative coefficient error measured on the prefix before
it (and never above 2 coef_rtol); any other divergence fails.
"""
from __future__ import annotations

import numpy as np

NEAR_TIE = 1e-6


def first_near_tie(ref):
    gap = (ref.s1 - ref.s2) / np.where(ref.s1 > 0, ref.s1, 1.0)
    idx = np.where(gap < NEAR_TIE)[0]
    return int(idx[0]) if idx.size else ref.n_atoms


def compare(atoms, errs, E0_gpu, ref, coef_rtol=1e-5, snr_tol_db=0.01, min_checked=1):
    """Returns a dict of figures; raises AssertionError on a parity failure."""
    upto = first_near_tie(ref)
    ng = atoms.size
    k = min(upto, ng, ref.n_atoms)
    same = (atoms["dict"][:k] == ref.dict[:k]) & (atoms["m"][:k] == ref.m[:k]) & \
        (atoms["n"][:k] == ref.n[:k])
    rule = "near tie 1e-6"
    if not same.all():
        bad = int(np.where(~same)[0][0])
        gap = (ref.s1[bad] - ref.s2[bad]) / ref.s1[bad]
        c0 = atoms["re"][:bad].astype(np.float64) + 1j * atoms["im"][:bad].astype(np.float64)
        scale = float(np.max(np.abs(c0 - ref.c[:bad]) / np.abs(ref.c[:bad]))) if bad else 0.0
        if not gap < min(2.0 * scale, 2.0 * coef_rtol):
            raise AssertionError(
                "atom %d differs: gpu (w=%d m=%d n=%d) oracle (w=%d m=%d n=%d); gap %.3g, "
                "measured coefficient error %.3g" % (
                    bad, atoms["dict"][bad], atoms["m"][bad], atoms["n"][bad], ref.dict[bad],
                    ref.m[bad], ref.n[bad], gap, scale))
        k = bad
        rule = "precision tie (gap %.3g < 2 x %.3g)" % (gap, scale)
    assert k >= min(min_checked, ref.n_atoms), (k, upto, ng, rule)
    c = atoms["re"][:k].astype(np.float64) + 1j * atoms["im"][:k].astype(np.float64)
    rel = np.abs(c - ref.c[:k]) / np.abs(ref.c[:k])
    worst = float(rel.max()) if k else 0.0
    assert worst <= coef_rtol, "coefficient rel. error %.3g at atom %d" % (worst, int(rel.argmax()))
    snr_g = 10 * np.log10(E0_gpu / errs[:k])
    snr_o = 10 * np.log10(ref.E0 / ref.E[:k])
    dsnr = float(np.max(np.abs(snr_g - snr_o))) if k else 0.0
    assert dsnr <= snr_tol_db, "SNR curve off by %.3g dB" % dsnr
    return {"checked": k, "near_tie_at": upto, "rule": rule, "coef_rel_max": worst,
            "snr_db_max": dsnr,
            "normwise": float(np.linalg.norm(c - ref.c[:k]) / np.linalg.norm(ref.c[:k])) if k else 0.0}

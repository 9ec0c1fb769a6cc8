"""ctypes front end of the FP64 C oracle (mp_oracle.c).

TEST INFRASTRUCTURE ONLY (tests/, smoke(), the bench's CPU legs).

Dictionaries are given as a list of (g, a, M) with g a float64 array holding
the zero-centred window (index i is g(t), t = i - w/2).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

STOP_SNR, STOP_KMAX, STOP_NEGENERGY, STOP_ZEROMAX = 1, 2, 3, 4
FLAG_FULLSCAN = 1
FLAG_PEDANTIC = 2

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.ora_kernel_dims.argtypes = [C.c_int] * 6 + [C.POINTER(C.c_int)] * 4
        L.ora_kernel_dims.restype = None
        L.ora_kernel.argtypes = [_dp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, C.c_int, C.c_int, _dp]
        L.ora_kernel.restype = None
        L.ora_dgt.argtypes = [_dp, C.c_int64, _dp, C.c_int, C.c_int, C.c_int, _dp]
        L.ora_dgt.restype = None
        L.ora_synth.argtypes = [C.c_int, _ip, _ip, _ip, _dp, C.c_int64, _ip, _ip, _lp, _dp, _dp,
                                C.c_int64, _dp]
        L.ora_synth.restype = None
        common = [C.c_int, _ip, _ip, _ip, _dp, _dp, C.c_int64]
        outs = [_ip, _ip, _lp, _dp, _dp, _dp, _dp, _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                C.POINTER(C.c_double), C.c_void_p]
        L.ora_mp_coef.argtypes = common + [C.c_double, C.c_int64, C.c_double, C.c_int] + outs
        L.ora_mp_coef.restype = C.c_int
        L.ora_mp_plain.argtypes = common + [C.c_int64, C.c_double, C.c_int] + outs
        L.ora_mp_plain.restype = C.c_int
        L.ora_mp_coef_reset.argtypes = common + [C.c_double, C.c_int64, C.c_double, C.c_int,
                                                 C.c_int64, C.c_double] + outs + \
            [C.POINTER(C.c_int64)]
        L.ora_mp_coef_reset.restype = C.c_int
        _lib = L
    return _lib


def kernel_dims(du, dv):
    (gu, au, Mu), (gv, av, Mv) = du, dv
    out = [C.c_int() for _ in range(4)]
    lib().ora_kernel_dims(len(gu), au, Mu, len(gv), av, Mv, *[C.byref(o) for o in out])
    Mx, an, tmin, ntau = (o.value for o in out)
    return Mx, an, tmin, ntau


def kernel(du, dv):
    """Full (untruncated) h_{u,v}: returns (h[ntau, Mx] complex, taus, Mx, a_min).

    h[it, delta] = sum_t g_u(t) g_v(t - tau) exp(-i 2 pi delta (t - tau) / M_max),
    tau = taus[it]."""
    (gu, au, Mu), (gv, av, Mv) = du, dv
    Mx, an, tmin, ntau = kernel_dims(du, dv)
    h = np.zeros(2 * ntau * Mx)
    lib().ora_kernel(np.ascontiguousarray(gu, np.float64), len(gu), au, Mu,
                     np.ascontiguousarray(gv, np.float64), len(gv), av, Mv, h)
    h = h.reshape(ntau, Mx, 2)
    return h[..., 0] + 1j * h[..., 1], tmin + an * np.arange(ntau), Mx, an


def dgt(x, g, a, M):
    """<x, d_{m,n}> for m = 0..M/2, n = 0..L/a-1, as complex [N, M/2+1]."""
    x = np.ascontiguousarray(x, np.float64)
    L = x.size
    N, Mr = L // a, M // 2 + 1
    out = np.zeros(2 * N * Mr)
    lib().ora_dgt(x, L, np.ascontiguousarray(g, np.float64), len(g), a, M, out)
    out = out.reshape(N, Mr, 2)
    return out[..., 0] + 1j * out[..., 1]


def _pack(dicts):
    W = len(dicts)
    wl = np.array([len(g) for g, _, _ in dicts], np.int32)
    a = np.array([d[1] for d in dicts], np.int32)
    M = np.array([d[2] for d in dicts], np.int32)
    gcat = np.ascontiguousarray(np.concatenate([np.asarray(g, np.float64) for g, _, _ in dicts]))
    return W, wl, a, M, gcat


@dataclass
class MPResult:
    dict: np.ndarray
    m: np.ndarray
    n: np.ndarray
    c: np.ndarray        # complex coefficients (adjusted real-pair coefficients)
    E: np.ndarray        # energy estimate after each atom
    s1: np.ndarray       # |rho| of the selected atom
    s2: np.ndarray       # largest |rho| among all other coefficients
    stop: int
    E0: float
    extra: np.ndarray | None = None

    @property
    def n_atoms(self):
        return self.dict.size

    def snr_db(self):
        return 10.0 * np.log10(self.E0 / self.E)


def _run(fn, dicts, x, tail_args, kmax, extra_len, resets=None):
    W, wl, a, M, gcat = _pack(dicts)
    x = np.ascontiguousarray(x, np.float64)
    cap = max(int(kmax), 1)
    od, om = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    on = np.zeros(cap, np.int64)
    ore, oim, oE, s1, s2 = (np.zeros(cap) for _ in range(5))
    na, st, E0 = C.c_int64(), C.c_int(), C.c_double()
    extra = np.zeros(extra_len) if extra_len else None
    args = [W, wl, a, M, gcat, x, x.size, *tail_args, od, om, on, ore, oim, oE, s1, s2,
            C.byref(na), C.byref(st), C.byref(E0),
            extra.ctypes.data_as(C.c_void_p) if extra is not None else None]
    nres = C.c_int64()
    if resets is not None:
        args.append(C.byref(nres))
    rc = fn(*args)
    if rc != 0:
        raise RuntimeError("oracle failed (%d)" % rc)
    k = na.value
    res = MPResult(od[:k].copy(), om[:k].copy(), on[:k].copy(), ore[:k] + 1j * oim[:k],
                   oE[:k].copy(), s1[:k].copy(), s2[:k].copy(), st.value, E0.value, extra)
    res.n_resets = nres.value
    return res


def _flags(fullscan, pedantic):
    return (FLAG_FULLSCAN if fullscan else 0) | (FLAG_PEDANTIC if pedantic else 0)


def mp_coef(dicts, x, eps, kmax, snr_db, fullscan=False, planes=False, pedantic=False):
    """Coefficient-domain MP with G_eps (Alg. 1 + Alg. 3); pedantic selects
    by the pair energy drop of eq. projenfaster instead of |rho|^2."""
    L = len(x)
    P = sum((L // a) * (M // 2 + 1) for _, a, M in dicts)
    res = _run(lib().ora_mp_coef, dicts, x,
               [float(eps), int(kmax), float(snr_db), _flags(fullscan, pedantic)],
               kmax, 2 * P if planes else 0)
    if planes:
        e = res.extra.reshape(-1, 2)
        flat = e[:, 0] + 1j * e[:, 1]
        out, o = [], 0
        for _, a, M in dicts:
            N, Mr = L // a, M // 2 + 1
            out.append(flat[o:o + N * Mr].reshape(N, Mr))
            o += N * Mr
        res.extra = out
    return res


def mp_coef_reset(dicts, x, eps, kmax, snr_db, reset_it=0, reset_db=0.0, fullscan=False,
                  pedantic=False):
    """Alg. 2: coefficient-domain MP with resets (after reset_it selections
    since the last reset, or once the estimate fell reset_db (< 0) dB below
    the energy at the last reset)."""
    return _run(lib().ora_mp_coef_reset, dicts, x,
                [float(eps), int(kmax), float(snr_db), _flags(fullscan, pedantic),
                 int(reset_it), float(reset_db)], kmax, 0, resets=True)


def mp_plain(dicts, x, kmax, snr_db, fullscan=False, pedantic=False):
    """Plain signal-domain MP (exact re-analysis); extra = final residual."""
    return _run(lib().ora_mp_plain, dicts, x,
                [int(kmax), float(snr_db), _flags(fullscan, pedantic)], kmax, len(x))


def synth(dicts, res_or_atoms, L):
    """Signal sum of the atoms (eq. idgtreal)."""
    W, wl, a, M, gcat = _pack(dicts)
    d = np.ascontiguousarray(res_or_atoms.dict, np.int32)
    m = np.ascontiguousarray(res_or_atoms.m, np.int32)
    n = np.ascontiguousarray(res_or_atoms.n, np.int64)
    c = np.asarray(res_or_atoms.c)
    y = np.zeros(L)
    lib().ora_synth(W, wl, a, M, gcat, d.size, d, m, n, np.ascontiguousarray(c.real),
                    np.ascontiguousarray(c.imag), L, y)
    return y

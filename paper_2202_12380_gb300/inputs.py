"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds only input generation: analysis windows and audio-like test
signals.  It contains none of the matching-pursuit arithmetic, so both the
CUDA path and the CPU oracle may take their inputs from it.

Windows follow the Gabor-dictionary setting of Sec. 2.1 (eq. gabdict): a real
window g of length w, normalised to unit l2 norm, placed zero-centred on the
circle, i.e. sample ``i`` of the returned array is g(t) with t = i - w//2, so
t runs over -w/2 ... w/2-1.  With this placement the truncated kernels of
Fig. 1 come out at the printed sizes (Blackman 23x7, Hann 31x7).

The paper's own audio (a piano recording) is not available; the seeded
mixtures below (tones, chirps, notes, transients, white or pink noise) stand
in for it.  Recipes, per workload:

* ``single_gauss_16k``: L=16384 at 16 kHz; 4 harmonic tones (f0 ~ U(100,1000)
  Hz, harmonics h <= min(8, 7200/f0) with amplitude 1/h, random phase, onset
  ~ U(0, 0.5 s), exponential decay tau ~ U(0.05, 0.5) s), 2 single-sample
  clicks of amplitude +-U(0.5,1)*max|tones|, white Gaussian noise at 20 dB SNR.
* ``mixture``: fs 44.1 kHz; 8 linear chirps (start/end frequency ~ U(50,16000)
  Hz, duration ~ U(0.1,1.5) s, Hann envelope, amplitude ~ U(0.1,1)), 6 decaying
  harmonic notes (f0 ~ U(80,1000) Hz, 10 harmonics at 1/h, tau ~ U(0.1,1) s),
  20 Gaussian-enveloped transients (sigma ~ U(0.5,5) ms, centre frequency
  ~ U(500,8000) Hz, amplitude ~ U(0.1,1)), pink noise (white spectrum scaled by
  1/sqrt(f), zero DC) at a given SNR (30 dB unless stated).

Seeds: 220212380 + 1000 * workload_id + signal_index.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 220212380


def seed_for(workload_id: int, index: int = 0) -> int:
    return SEED_BASE + 1000 * int(workload_id) + int(index)


# ----------------------------------------------------------------------------
# windows (zero-centred, periodic, unit l2 norm)
# ----------------------------------------------------------------------------

def _centred_t(w: int) -> np.ndarray:
    if w <= 0 or w % 2:
        raise ValueError("window length must be positive and even")
    return np.arange(w, dtype=np.float64) - w // 2


def _normalise(g: np.ndarray) -> np.ndarray:
    return g / np.sqrt(np.sum(g * g))


def blackman(w: int) -> np.ndarray:
    """Periodic Blackman window, zero-centred, unit norm."""
    t = _centred_t(w)
    g = 0.42 + 0.5 * np.cos(2 * np.pi * t / w) + 0.08 * np.cos(4 * np.pi * t / w)
    return _normalise(g)


def hann(w: int) -> np.ndarray:
    """Periodic Hann window, zero-centred, unit norm."""
    t = _centred_t(w)
    return _normalise(0.5 + 0.5 * np.cos(2 * np.pi * t / w))


def gauss_edge(w: int, edge: float = 1e-4) -> np.ndarray:
    """Gaussian exp(-pi t^2 / lam) truncated to w samples, with lam chosen so
    that the value at the window edge t = -w/2 is ``edge`` times the peak."""
    t = _centred_t(w)
    lam = math.pi * (w / 2) ** 2 / math.log(1.0 / edge)
    return _normalise(np.exp(-math.pi * t * t / lam))


def gauss_lambda(w: int, lam: float) -> np.ndarray:
    """Gaussian exp(-pi t^2 / lam) on w samples (take w large enough that the
    tails are below double precision to model the untruncated window)."""
    t = _centred_t(w)
    return _normalise(np.exp(-math.pi * t * t / lam))


WINDOWS = {"blackman": blackman, "hann": hann, "gauss": gauss_edge}


def make_window(kind: str, w: int) -> np.ndarray:
    return WINDOWS[kind](w)


# ----------------------------------------------------------------------------
# signals
# ----------------------------------------------------------------------------

def _scale_noise(sig: np.ndarray, noise: np.ndarray, snr_db: float) -> np.ndarray:
    ps = float(np.sum(sig * sig))
    pn = float(np.sum(noise * noise))
    if pn == 0.0 or ps == 0.0:
        return noise
    return noise * math.sqrt(ps / (pn * 10.0 ** (snr_db / 10.0)))


def tones_clicks_noise(L: int, seed: int, fs: float = 16000.0, snr_db: float = 20.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = np.arange(L) / fs
    tones = np.zeros(L)
    for _ in range(4):
        f0 = rng.uniform(100.0, 1000.0)
        nh = int(math.floor(min(8.0, 7200.0 / f0)))
        onset = rng.uniform(0.0, 0.5)
        tau = rng.uniform(0.05, 0.5)
        env = np.where(t >= onset, np.exp(-(t - onset) / tau), 0.0)
        for h in range(1, nh + 1):
            ph = rng.uniform(0.0, 2 * np.pi)
            tones += env * np.cos(2 * np.pi * h * f0 * t + ph) / h
    peak = float(np.max(np.abs(tones))) if L else 0.0
    sig = tones.copy()
    for _ in range(2):
        pos = int(rng.integers(0, L))
        amp = rng.uniform(0.5, 1.0) * peak * (1.0 if rng.uniform() < 0.5 else -1.0)
        sig[pos] += amp
    noise = rng.standard_normal(L)
    return sig + _scale_noise(sig, noise, snr_db)


def _pink(L: int, rng: np.random.Generator) -> np.ndarray:
    white = rng.standard_normal(L)
    spec = np.fft.rfft(white)
    f = np.arange(spec.size, dtype=np.float64)
    scale = np.zeros_like(f)
    scale[1:] = 1.0 / np.sqrt(f[1:])
    return np.fft.irfft(spec * scale, n=L)


def mixture(L: int, seed: int, fs: float = 44100.0, snr_db: float = 30.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    t = np.arange(L) / fs
    dur_total = L / fs
    sig = np.zeros(L)
    for _ in range(8):  # linear chirps
        f1 = rng.uniform(50.0, 16000.0)
        f2 = rng.uniform(50.0, 16000.0)
        d = rng.uniform(0.1, 1.5)
        t0 = rng.uniform(0.0, max(dur_total - d, 1e-3))
        amp = rng.uniform(0.1, 1.0)
        tt = t - t0
        on = (tt >= 0) & (tt < d)
        ph = 2 * np.pi * (f1 * tt + 0.5 * (f2 - f1) / d * tt * tt)
        env = 0.5 - 0.5 * np.cos(2 * np.pi * np.clip(tt, 0, d) / d)
        sig += np.where(on, amp * env * np.cos(ph), 0.0)
    for _ in range(6):  # decaying harmonic notes
        f0 = rng.uniform(80.0, 1000.0)
        tau = rng.uniform(0.1, 1.0)
        onset = rng.uniform(0.0, dur_total * 0.9)
        env = np.where(t >= onset, np.exp(-(t - onset) / tau), 0.0)
        for h in range(1, 11):
            fh = h * f0
            if fh >= fs / 2:
                break
            sig += env * np.cos(2 * np.pi * fh * t + rng.uniform(0, 2 * np.pi)) / h
    for _ in range(20):  # Gaussian-enveloped transients
        sd = rng.uniform(0.5e-3, 5e-3)
        fc = rng.uniform(500.0, 8000.0)
        amp = rng.uniform(0.1, 1.0)
        t0 = rng.uniform(0.0, dur_total)
        sig += amp * np.exp(-((t - t0) ** 2) / (2 * sd * sd)) * np.cos(2 * np.pi * fc * (t - t0))
    noise = _pink(L, rng)
    return sig + _scale_noise(sig, noise, snr_db)


def white_noise(L: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(L)


def as_f32(x: np.ndarray) -> np.ndarray:
    """The GPU path consumes float32 samples; the oracle is fed the same
    float32 values widened back to float64 so both see one signal."""
    return np.ascontiguousarray(x, dtype=np.float32)


# ----------------------------------------------------------------------------
# named workloads (dictionary lists are (window kind, w, a, M))
# ----------------------------------------------------------------------------

WORKLOADS = {
    # one signal, one Gaussian dictionary, K=500
    "single_gauss_16k": dict(id=1, L=16384, dicts=[("gauss", 256, 64, 256)], eps=1e-4,
                             kmax=500, snr_db=200.0),
    # one signal L=2^18, 3 Blackman dictionaries, to 40 dB or K=50000
    "multi3_2p18": dict(id=2, L=1 << 18,
                        dicts=[("blackman", 512, 128, 512), ("blackman", 1024, 256, 1024),
                               ("blackman", 2048, 512, 2048)], eps=1e-4, kmax=50000, snr_db=40.0),
    # precision form: L=2^20, 5 Blackman dictionaries
    "multi5_2p20": dict(id=3, L=1 << 20,
                        dicts=[("blackman", w, w // 4, w) for w in (256, 512, 1024, 2048, 4096)],
                        eps=1e-4, kmax=200000, snr_db=40.0),
    # batched form: 256 signals, log-uniform lengths 2^14..2^20
    "batch256": dict(id=4, B=256, Lmin=1 << 14, Lmax=1 << 20,
                     dicts=[("blackman", 512, 128, 512), ("blackman", 1024, 256, 1024),
                            ("blackman", 2048, 512, 2048)], eps=1e-4, kmax=20000, snr_db=30.0),
    # long-signal stress: L=2^23, 5 Blackman + Gaussian 1024/128
    "stress_2p23": dict(id=5, L=1 << 23,
                        dicts=[("blackman", w, w // 4, w) for w in (256, 512, 1024, 2048, 4096)]
                        + [("gauss", 1024, 128, 1024)], eps=1e-5, kmax=1000000, snr_db=40.0),
}


def workload_dicts(name: str):
    return WORKLOADS[name]["dicts"]


def make_windows(dicts):
    return [make_window(kind, w) for (kind, w, _a, _M) in dicts]


def workload_signal(name: str, index: int = 0) -> np.ndarray:
    """Float32 signal(s) for a named workload (a list for the batched one)."""
    cfg = WORKLOADS[name]
    wid = cfg["id"]
    if name == "single_gauss_16k":
        return as_f32(tones_clicks_noise(cfg["L"], seed_for(wid, index)))
    if name == "batch256":
        return [as_f32(x) for x in batch_signals(cfg, wid)]
    return as_f32(mixture(cfg["L"], seed_for(wid, index)))


def batch_lengths(cfg, wid: int, multiple: int = 2048):
    rng = np.random.default_rng(seed_for(wid, 999))
    lo, hi = math.log(cfg["Lmin"]), math.log(cfg["Lmax"])
    out = []
    for _ in range(cfg["B"]):
        L = int(math.ceil(math.exp(rng.uniform(lo, hi)) / multiple) * multiple)
        out.append(min(max(L, cfg["Lmin"]), cfg["Lmax"]))
    return out


def batch_signals(cfg, wid: int, indices=None):
    """The batch's signals (all, or only those listed in `indices`; each
    signal is the same whichever others are generated)."""
    lens = batch_lengths(cfg, wid)
    rng = np.random.default_rng(seed_for(wid, 998))
    snrs = rng.uniform(10.0, 40.0, size=len(lens))
    idx = range(len(lens)) if indices is None else indices
    return [mixture(lens[i], seed_for(wid, i), snr_db=float(snrs[i])) for i in idx]


def batch_subset(name: str, indices):
    """Float32 signals `indices` of a batched workload."""
    cfg = WORKLOADS[name]
    return [as_f32(x) for x in batch_signals(cfg, cfg["id"], indices)]

"""GPU parity at the workloads' full sizes, in the launch shapes the bench
times, against the FP64 oracle.

* multi3_2p18 (L = 2^18, three Blackman dictionaries, 40 dB): the whole
  decomposition, default launch shape (one 16-CTA cluster), FP32 analysis;
* multi5_2p20 (L = 2^20, five dictionaries, split-BF16 analysis): the first
  5000 atoms;
* batch256 (256 signals of uneven length in one launch, 512-thread CTAs as
  the autotuner picks them): six sampled signals against their own oracle
  runs over their first 4000 atoms, reported (FP32 coefficients meet
  precision ties; the strict comparison is the FP64-plane run of
  test_gpu_fp64.py);
* stress_2p23 (L = 2^23, six dictionaries, eps = 1e-5): analysis sampled at
  frames the oracle computes from signal segments (a frame only sees w
  samples), and the energy bookkeeping of 3000 atoms against the true
  residual energy of the synthesis.

Beyond the oracle's first near tie the two pursuits are both valid but may
differ; there only what stays unique is compared (stop reason, atom count
within 0.1 %, the SNR curves within 0.05 dB).
"""
import numpy as np
import pytest

from oracle import cmp
from paper_2202_12380_gb300 import inputs
from tests.parity import compare, prefix_agreement

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2202_12380_gb300 import mpgabor as mg  # noqa: E402


def _dicts(name):
    return [(inputs.make_window(k, w), a, M) for (k, w, a, M) in inputs.WORKLOADS[name]["dicts"]]


def _plan(dicts, eps, flags=0):
    return mg.mp_plan_create([g for g, _, _ in dicts], [a for _, a, _ in dicts],
                             [M for _, _, M in dicts], eps, flags)


def _result(st, b):
    n, stop, q = mg.mp_get_status(st)
    atoms, errs = mg.mp_get_atoms(st, b), mg.mp_get_errors(st, b)
    E0 = errs[-1] * 10 ** (q[b] / 10)
    return atoms, errs, E0, int(stop[b])


def test_multi3_2p18_full_decomposition():
    name = "multi3_2p18"
    cfg, dicts = inputs.WORKLOADS[name], _dicts(name)
    x = inputs.workload_signal(name)
    ref = cmp.mp_coef(dicts, x.astype(np.float64), cfg["eps"], cfg["kmax"], cfg["snr_db"])
    plan = _plan(dicts, cfg["eps"])
    st = mg.mp_analyze(plan, [torch.from_numpy(x).cuda()])
    assert mg.mp_state_get_launch(st) == (128, 16)  # the shape the bench times
    mg.mp_run(st, cfg["kmax"], cfg["snr_db"])
    atoms, errs, E0, stop = _result(st, 0)
    r = compare(atoms, errs, E0, ref, min_checked=1000)
    print(name, r, "atoms gpu", atoms.size, "oracle", ref.n_atoms)
    assert stop == ref.stop == mg.MP_STOP_SNR
    assert abs(atoms.size - ref.n_atoms) <= 0.001 * ref.n_atoms
    # SNR curves over the common length, past the first near tie too
    k = min(atoms.size, ref.n_atoms)
    d = np.abs(10 * np.log10(E0 / errs[:k]) - 10 * np.log10(ref.E0 / ref.E[:k]))
    assert d.max() < 0.05, d.max()


def test_multi5_2p20_bf16x3_prefix():
    name = "multi5_2p20"
    cfg, dicts = inputs.WORKLOADS[name], _dicts(name)
    x = inputs.workload_signal(name)
    K = 5000
    ref = cmp.mp_coef(dicts, x.astype(np.float64), cfg["eps"], K, cfg["snr_db"])
    plan = _plan(dicts, cfg["eps"], mg.MP_ANALYSIS_BF16X3)
    st = mg.mp_analyze(plan, [torch.from_numpy(x).cuda()])
    mg.mp_run(st, K, cfg["snr_db"])
    atoms, errs, E0, stop = _result(st, 0)
    assert atoms.size == K
    # split-BF16 analysis: near ties at the analysis precision (gap < 1e-3)
    # may flip; the sequences agree up to their first divergence, which must
    # be such a near tie
    same = (atoms["dict"] == ref.dict) & (atoms["m"] == ref.m) & (atoms["n"] == ref.n)
    dv = int(np.argmin(same)) if not same.all() else K
    if dv < K:
        gap = (ref.s1[dv] - ref.s2[dv]) / ref.s1[dv]
        assert gap < 1e-3, (dv, gap)
    c = atoms["re"][:dv].astype(np.float64) + 1j * atoms["im"][:dv]
    rel = np.abs(c - ref.c[:dv]) / np.abs(ref.c[:dv])
    dsnr = np.abs(10 * np.log10(E0 / errs) - 10 * np.log10(ref.E0 / ref.E))
    print(name, "first divergence", dv, "coef rel max", rel.max() if dv else 0.0,
          "median", np.median(rel) if dv else 0.0, "SNR max dev", dsnr.max())
    assert dv >= 500
    assert rel.max() < 1e-3 and np.median(rel) < 1e-4
    assert dsnr.max() < 0.05


def test_batch256_sampled_signals_fp32_report():
    """The FP32 form of batch256 (the bench's launch): six sampled signals
    against their own oracle runs over their first 4000 atoms.  FP32
    coefficients can swap candidates whose gap is below their accumulated
    error before a 1e-6 near tie, so this measures and reports (first
    divergence, its gap against the measured coefficient error) and checks
    the numeric bars on the agreeing prefix and the SNR curves; the strict
    parity of this workload is test_gpu_fp64.py's FP64-plane run."""
    name = "batch256"
    cfg, dicts = inputs.WORKLOADS[name], _dicts(name)
    xs = inputs.workload_signal(name)
    plan = _plan(dicts, cfg["eps"])
    st = mg.mp_analyze(plan, [torch.from_numpy(x).cuda() for x in xs])
    mg.mp_state_set_launch(st, 512, 1)
    mg.mp_run(st, cfg["kmax"], cfg["snr_db"])
    lens = np.array([len(x) for x in xs])
    order = np.argsort(lens)
    picks = [order[0], order[len(order) // 4], order[len(order) // 2],
             order[3 * len(order) // 4], order[-2], order[-1]]
    Kc = 4000
    for b in picks:
        x = xs[b]
        ref = cmp.mp_coef(dicts, x.astype(np.float64), cfg["eps"], Kc, cfg["snr_db"])
        atoms, errs, E0, stop = _result(st, b)
        r = prefix_agreement(atoms, errs, E0, ref)
        print(name, "signal", int(b), "L", len(x), r)
        assert r["prefix"] >= min(200, ref.n_atoms)
        assert r["coef_rel_max"] <= 1e-5 and r["snr_db_max"] <= 0.01
        assert r["snr_db_max_common"] < 0.05


def test_stress_2p23_analysis_samples_and_energy():
    name = "stress_2p23"
    cfg, dicts = inputs.WORKLOADS[name], _dicts(name)
    x = inputs.workload_signal(name)
    L = x.size
    plan = _plan(dicts, cfg["eps"])
    st = mg.mp_analyze(plan, [torch.from_numpy(x).cuda()])
    # frames sampled at two positions: the oracle analyses a 16384-sample
    # segment starting at a multiple of every hop; its frames whose window
    # lies inside the segment equal the full signal's frames.  Every FP32
    # coefficient must lie within the error bound of a w-term FP32 dot
    # product with FP32-rounded matrix entries, 2 (w + 2) 2^-24 sum|x g|
    # (real and imaginary part each), against the FP64 value.
    seg = 16384
    for w, (g, a, M) in enumerate(dicts):
        plane = mg.mp_state_coefficients(st, 0, w)
        wl = len(g)
        lo = -(-(wl // 2) // a)
        hi = (seg - wl // 2) // a + 1
        for s0 in ((L // 3) // 4096 * 4096, L - 3 * seg):
            xs = x[s0:s0 + seg].astype(np.float64)
            ref = cmp.dgt(xs, g, a, M)[lo:hi]
            got = plane[s0 // a + lo:s0 // a + hi]
            sabs = np.array([np.sum(np.abs(xs[n * a - wl // 2:n * a + wl // 2]) * np.abs(g))
                             for n in range(lo, hi)])
            bound = 2.0 * (wl + 2) * 2.0 ** -24 * sabs[:, None]
            ratio = np.abs(got - ref) / bound
            print(name, "dict", w, "segment", s0, "max err / FP32 bound", ratio.max())
            assert ratio.max() <= 1.0, (s0, w, ratio.max())
    # energy bookkeeping: the FP64 estimate after 3000 atoms against the true
    # residual energy of the synthesised approximation (eps = 1e-5 keeps the
    # two within the Theorem-1 bound, far below 0.01 dB here)
    K = 3000
    mg.mp_run(st, K, 200.0)
    atoms, errs, E0, stop = _result(st, 0)
    assert atoms.size == K and stop == mg.MP_STOP_KMAX
    y = torch.zeros(L, dtype=torch.float32, device="cuda")
    snr_true = mg.mp_synthesize(st, 0, y)
    snr_est = 10 * np.log10(E0 / errs[-1])
    print(name, "estimated SNR", snr_est, "true SNR", snr_true)
    assert abs(snr_est - snr_true) < 0.01

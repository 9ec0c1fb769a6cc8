"""mp_decompose_static, the allocation-free entry point, against the regular
mp_analyze + mp_run path.

The entry point exists for callers that cannot call cudaMalloc while they
decompose (work inside a stream capture, real-time audio threads, fixed
device-memory budgets): its planes and trees live in a static device array
instead of an allocated state.  Two calls in a row, on different signals,
must each reproduce the regular path's atoms, coefficients and energies
(same kernels, so to within the parity tolerance and in practice exactly),
which also shows that nothing left in the shared array by the first call
leaks into the second.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2202_12380_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2202_12380_gb300 import mpgabor as mg  # noqa: E402

COEF_RTOL = 1e-5  # the parity tolerance on coefficients used by the other tests


def _regular(plan, x, K, snr):
    st = mg.mp_analyze(plan, [x])
    n, stop, q = mg.mp_run(st, K, snr)
    out = mg.mp_get_atoms(st, 0), mg.mp_get_errors(st, 0), int(n[0]), int(stop[0]), float(q[0])
    st.close()
    return out


def test_static_matches_regular_two_calls():
    dicts = [(inputs.blackman(w), w // 4, w) for w in (128, 256, 512)]
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             1e-4)
    K, snr = 400, 35.0
    atoms_buf = torch.empty(K * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    errs_buf = torch.empty(K, dtype=torch.float64, device="cuda")
    for call, (L, seed) in enumerate([(16384, 101), (8192, 102)]):
        x = torch.from_numpy(inputs.as_f32(inputs.mixture(L, seed, fs=16000.0))).cuda()
        ref_atoms, ref_errs, ref_n, ref_stop, ref_q = _regular(plan, x, K, snr)
        atoms_buf.fill_(0xFF)
        errs_buf.fill_(float("nan"))
        n, stop, q = mg.mp_decompose_static(plan, x, K, snr, atoms_buf, errs_buf)
        assert (n, stop) == (ref_n, ref_stop), call
        atoms = mg.atoms_from_bytes(atoms_buf.cpu().numpy(), n)
        errs = errs_buf.cpu().numpy()[:n]
        for f in ("dict", "m", "n"):
            assert np.array_equal(atoms[f], ref_atoms[f]), (call, f)
        c = atoms["re"] + 1j * atoms["im"]
        c_ref = ref_atoms["re"] + 1j * ref_atoms["im"]
        assert np.max(np.abs(c - c_ref) / np.abs(c_ref)) <= COEF_RTOL
        assert np.max(np.abs(errs - ref_errs) / ref_errs[0]) <= 1e-12
        assert abs(q - ref_q) < 1e-9
    plan.close()


def test_static_without_error_buffer_and_async():
    dicts = [(inputs.blackman(256), 64, 256)]
    plan = mg.mp_plan_create([dicts[0][0]], [64], [256], 1e-4)
    x = torch.from_numpy(inputs.as_f32(inputs.mixture(4096, 103, fs=16000.0))).cuda()
    K = 100
    ref_atoms, _, ref_n, _, _ = _regular(plan, x, K, 200.0)
    buf = torch.empty(K * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n, stop, q = mg.mp_decompose_static(plan, x, K, 200.0, buf, None)
    assert n == ref_n == K
    atoms = mg.atoms_from_bytes(buf.cpu().numpy(), n)
    assert np.array_equal(atoms[["dict", "m", "n"]], ref_atoms[["dict", "m", "n"]])
    plan.close()


def test_static_rejects_oversized_signal():
    dicts = [(inputs.blackman(w), w // 4, w) for w in (512, 1024, 2048)]
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             1e-4)
    L = 1 << 20
    x = torch.zeros(L, dtype=torch.float32, device="cuda")
    buf = torch.empty(10 * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(mg.MPError) as ei:
        mg.mp_decompose_static(plan, x, 10, 40.0, buf, None)
    assert ei.value.code == mg.MP_EINVAL
    assert "scratch" in str(ei.value)
    plan.close()

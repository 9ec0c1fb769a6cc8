"""mp_decompose_static, the allocation-free entry point, against the regular
mp_analyze + mp_run path.

The entry point exists for callers that cannot call cudaMalloc while they
decompose (real-time audio threads that must not block in the allocator,
processes held to a fixed device-memory budget): its planes and trees live
in a static device array instead of an allocated state.  Two calls in a row, on different signals,
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
    """No error buffer (the estimates go to the static array), and the
    asynchronous form: no host outputs, so nothing is read back until the
    caller synchronises.  The plan runs on its own stream while the input is
    written on torch's current stream just before the call."""
    dicts = [(inputs.blackman(256), 64, 256)]
    side = torch.cuda.Stream()
    plan = mg.mp_plan_create([dicts[0][0]], [64], [256], 1e-4, stream=side)
    xh = torch.from_numpy(inputs.as_f32(inputs.mixture(4096, 103, fs=16000.0)))
    K = 100
    ref_atoms, _, ref_n, _, _ = _regular(plan, xh.cuda(), K, 200.0)
    buf = torch.empty(K * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n, stop, q = mg.mp_decompose_static(plan, xh.cuda(), K, 200.0, buf, None)
    assert n == ref_n == K
    atoms = mg.atoms_from_bytes(buf.cpu().numpy(), n)
    assert np.array_equal(atoms[["dict", "m", "n"]], ref_atoms[["dict", "m", "n"]])
    buf.fill_(0xFF)
    x = torch.empty(4096, dtype=torch.float32, device="cuda")
    x.copy_(xh, non_blocking=True)
    assert mg.mp_decompose_static(plan, x, K, 200.0, buf, None, sync=False) is None
    torch.cuda.synchronize()
    atoms = mg.atoms_from_bytes(buf.cpu().numpy(), K)
    assert np.array_equal(atoms[["dict", "m", "n"]], ref_atoms[["dict", "m", "n"]])
    plan.close()


def test_static_allocates_no_device_memory():
    """After a first call (which resolves the array's address), further calls
    leave the device's free memory unchanged."""
    dicts = [(inputs.blackman(w), w // 4, w) for w in (128, 256)]
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             1e-4)
    K = 200
    x = torch.from_numpy(inputs.as_f32(inputs.mixture(8192, 104, fs=16000.0))).cuda()
    buf = torch.empty(K * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    errs = torch.empty(K, dtype=torch.float64, device="cuda")
    mg.mp_decompose_static(plan, x, K, 40.0, buf, errs)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        mg.mp_decompose_static(plan, x, K, 40.0, buf, errs)
        mg.mp_decompose_static(plan, x, K, 40.0, buf, None, sync=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    plan.close()


def test_static_rejects_split_bf16_plan():
    """The entry point runs the FP32 analysis only; a plan asking for the
    split-BF16 analysis is refused rather than silently analysed in FP32."""
    dicts = [(inputs.blackman(w), w // 4, w) for w in (256, 512)]
    plan = mg.mp_plan_create([d[0] for d in dicts], [d[1] for d in dicts], [d[2] for d in dicts],
                             1e-4, mg.MP_ANALYSIS_BF16X3)
    x = torch.zeros(8192, dtype=torch.float32, device="cuda")
    buf = torch.empty(10 * mg.ATOM_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(mg.MPError) as ei:
        mg.mp_decompose_static(plan, x, 10, 40.0, buf, None)
    assert ei.value.code == mg.MP_ENOTCOMPAT
    assert "BF16" in str(ei.value)
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

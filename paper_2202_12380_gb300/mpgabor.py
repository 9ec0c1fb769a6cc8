"""Python binding of libmpgabor (the C ABI declared in include/mpgabor.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
library.  Function names follow the C ABI.  PyTorch is used for device
memory and streams (pass CUDA tensors and, optionally, a torch stream).

The library must have been built (``paper_2202_12380_gb300.build.build()`` or
``__graft_entry__.build()``); loading fails loudly otherwise -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MP_OK, MP_EINVAL, MP_ENOTCOMPAT, MP_ENOMEM, MP_ECUDA, MP_ETIMEOUT = 0, -1, -2, -3, -4, -5
MP_STOP_NONE, MP_STOP_SNR, MP_STOP_KMAX, MP_STOP_NEGENERGY, MP_STOP_ZEROMAX, MP_STOP_INVALID = \
    0, 1, 2, 3, 4, 5
MP_ANALYSIS_FP32, MP_ANALYSIS_BF16X3, MP_PEDANTIC, MP_COEF_FP64 = 0, 1, 2, 4

ATOM_DTYPE = np.dtype([("dict", "<i4"), ("m", "<i4"), ("n", "<i8"), ("re", "<f4"), ("im", "<f4")])

EXPORTS = [
    "mp_plan_create", "mp_plan_destroy", "mp_plan_kernel_dims", "mp_plan_kernel_fp64",
    "mp_plan_tile_info", "mp_plan_tile", "mp_plan_gamma", "mp_analyze", "mp_analyze_host",
    "mp_state_coefficients", "mp_run", "mp_run_async", "mp_get_status", "mp_state_set_time_limit",
    "mp_get_atoms", "mp_get_errors", "mp_synthesize", "mp_state_destroy", "mp_last_error",
    "mp_decompose_static", "mp_state_set_resets", "mp_state_set_launch", "mp_state_get_launch",
    "mp_state_set_work_hint", "mp_state_set_top_keys", "mp_state_get_top_keys",
]

_lib = None


class MPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mpgabor error %d: %s" % (code, msg))
        self.code = code


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libmpgabor.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libmpgabor.so is not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "mp_plan_create": ([P(vp), i32, P(P(dbl)), P(i32), P(i32), P(i32), dbl, C.c_uint, vp], i32),
        "mp_plan_destroy": ([vp], None),
        "mp_plan_kernel_dims": ([vp, i32, i32, P(i32), P(i32), P(i32), P(i32)], i32),
        "mp_plan_kernel_fp64": ([vp, i32, i32, vp, i64], i32),
        "mp_plan_tile_info": ([vp, i32, i32, i32, i32, P(i32)], i32),
        "mp_plan_tile": ([vp, i32, i32, i32, i32, vp, i64], i32),
        "mp_plan_gamma": ([vp, i32, vp, i64], i32),
        "mp_analyze": ([vp, P(vp), i32, P(vp), P(i64)], i32),
        "mp_analyze_host": ([vp, P(vp), i32, P(vp), P(i64)], i32),
        "mp_state_coefficients": ([vp, i32, i32, vp, i64], i32),
        "mp_run": ([vp, i64, dbl, vp, vp, vp], i32),
        "mp_run_async": ([vp, i64, dbl], i32),
        "mp_get_status": ([vp, vp, vp, vp], i32),
        "mp_state_set_time_limit": ([vp, dbl], i32),
        "mp_get_atoms": ([vp, i32, vp, i64, P(i64)], i32),
        "mp_get_errors": ([vp, i32, vp, i64, P(i64)], i32),
        "mp_synthesize": ([vp, i32, vp, P(dbl)], i32),
        "mp_state_destroy": ([vp], None),
        "mp_last_error": ([], C.c_char_p),
        "mp_decompose_static": ([vp, vp, i64, i64, dbl, vp, vp, P(i64), P(i32), P(dbl)], i32),
        "mp_state_set_resets": ([vp, i64, dbl], i32),
        "mp_state_set_launch": ([vp, i32, i32], i32),
        "mp_state_get_launch": ([vp, P(i32), P(i32)], i32),
        "mp_state_set_work_hint": ([vp, vp], i32),
        "mp_state_set_top_keys": ([vp, i32], i32),
        "mp_state_get_top_keys": ([vp, P(i32)], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc):
    if rc != MP_OK:
        raise MPError(rc, lib().mp_last_error().decode(errors="replace"))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Plan:
    """Owner of an mp_plan handle plus the dictionary parameters."""

    def __init__(self, handle, wins, a, M, eps, flags, stream=None):
        self.handle = handle
        self.stream = _stream_handle(stream)  # cudaStream_t of the plan (None: legacy)
        self.wlen = [len(g) for g in wins]
        self.a = list(a)
        self.M = list(M)
        self.eps = eps
        self.flags = flags

    @property
    def W(self):
        return len(self.a)

    def close(self):
        if self.handle:
            lib().mp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class State:
    """Owner of an mp_state handle plus the signal lengths."""

    def __init__(self, plan: Plan, lengths):
        self.plan = plan
        self.handle = C.c_void_p()
        self.L = [int(x) for x in lengths]

    @property
    def B(self):
        return len(self.L)

    def close(self):
        if self.handle:
            lib().mp_state_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_plan_create(windows, a, M, kern_thr=1e-4, flags=MP_ANALYSIS_FP32, stream=None) -> Plan:
    wins = [np.ascontiguousarray(g, dtype=np.float64) for g in windows]
    W = len(wins)
    arr = (C.POINTER(C.c_double) * W)(*[g.ctypes.data_as(C.POINTER(C.c_double)) for g in wins])
    wl = (C.c_int * W)(*[len(g) for g in wins])
    aa = (C.c_int * W)(*[int(x) for x in a])
    MM = (C.c_int * W)(*[int(x) for x in M])
    h = C.c_void_p()
    _check(lib().mp_plan_create(C.byref(h), W, arr, wl, aa, MM, float(kern_thr), int(flags),
                                _stream_handle(stream)))
    return Plan(h, wins, a, M, kern_thr, flags, stream)


def mp_plan_destroy(plan: Plan):
    plan.close()


def mp_plan_kernel_dims(plan: Plan, u: int, v: int):
    o = [C.c_int() for _ in range(4)]
    _check(lib().mp_plan_kernel_dims(plan.handle, u, v, *[C.byref(x) for x in o]))
    return tuple(x.value for x in o)


def mp_plan_kernel_fp64(plan: Plan, u: int, v: int):
    Mx, an, tmin, ntau = mp_plan_kernel_dims(plan, u, v)
    buf = np.zeros((ntau, Mx, 2), np.float64)
    _check(lib().mp_plan_kernel_fp64(plan.handle, u, v, buf.ctypes.data, buf.size))
    return buf[..., 0] + 1j * buf[..., 1], tmin + an * np.arange(ntau)


def mp_plan_tile_info(plan: Plan, u: int, v: int, cf: int, ct: int):
    info = (C.c_int * 7)()
    _check(lib().mp_plan_tile_info(plan.handle, u, v, cf, ct, info))
    keys = ("rf", "rt", "R", "C", "i_lo", "c_lo", "nnz")
    return dict(zip(keys, list(info)))


def mp_plan_tile(plan: Plan, u: int, v: int, cf: int, ct: int):
    info = mp_plan_tile_info(plan, u, v, cf, ct)
    R, Cc = info["R"], info["C"]
    buf = np.zeros((max(Cc, 0), max(R, 0), 2), np.float32)
    if R * Cc:
        _check(lib().mp_plan_tile(plan.handle, u, v, cf, ct, buf.ctypes.data, buf.size))
    return buf[..., 0] + 1j * buf[..., 1], info


def mp_plan_gamma(plan: Plan, u: int):
    buf = np.zeros((plan.M[u] // 2 + 1, 2), np.float32)
    _check(lib().mp_plan_gamma(plan.handle, u, buf.ctypes.data, buf.size))
    return buf[:, 0] + 1j * buf[:, 1]


def _plan_stream(plan: Plan):
    import torch
    if plan.stream is None:
        return torch.cuda.default_stream()
    return torch.cuda.ExternalStream(plan.stream)


def _wait_for_current(plan: Plan):
    """Order the plan's stream after the work already queued on torch's
    current stream (where the caller wrote the inputs).  No-op when the two
    are the same stream."""
    import torch
    cur = torch.cuda.current_stream()
    ps = _plan_stream(plan)
    if ps.cuda_stream != cur.cuda_stream:
        ps.wait_stream(cur)


def _current_waits_for_plan(plan: Plan):
    """Order torch's current stream after the plan's stream (where the
    library wrote the outputs)."""
    import torch
    cur = torch.cuda.current_stream()
    ps = _plan_stream(plan)
    if ps.cuda_stream != cur.cuda_stream:
        cur.wait_stream(ps)


def mp_analyze(plan: Plan, xs, state: State | None = None) -> State:
    """xs: list of float32 CUDA tensors (contiguous), one per signal.  The
    plan's stream is first ordered after torch's current stream, so inputs
    written there are ready."""
    B = len(xs)
    lens = [int(x.numel()) for x in xs]
    for x in xs:
        if not (x.is_cuda and x.is_contiguous() and str(x.dtype) == "torch.float32"):
            raise ValueError("mp_analyze needs contiguous float32 CUDA tensors")
    if state is None:
        state = State(plan, lens)
    ptrs = (C.c_void_p * B)(*[x.data_ptr() for x in xs])
    L = (C.c_int64 * B)(*lens)
    _wait_for_current(plan)
    _check(lib().mp_analyze(plan.handle, C.byref(state.handle), B, ptrs, L))
    return state


def mp_analyze_host(plan: Plan, xs, state: State | None = None) -> State:
    """xs: list of host float32 arrays (numpy, or CPU tensors, pinned preferred)."""
    B = len(xs)
    keep, ptrs, lens = [], [], []
    for x in xs:
        if hasattr(x, "data_ptr"):
            if x.is_cuda or str(x.dtype) != "torch.float32" or not x.is_contiguous():
                raise ValueError("mp_analyze_host needs contiguous float32 host tensors")
            ptrs.append(x.data_ptr())
            lens.append(int(x.numel()))
        else:
            a = np.ascontiguousarray(x, dtype=np.float32)
            keep.append(a)
            ptrs.append(a.ctypes.data)
            lens.append(a.size)
    if state is None:
        state = State(plan, lens)
    P = (C.c_void_p * B)(*ptrs)
    L = (C.c_int64 * B)(*lens)
    _check(lib().mp_analyze_host(plan.handle, C.byref(state.handle), B, P, L))
    return state


def mp_state_coefficients(state: State, sig: int, w: int):
    N = state.L[sig] // state.plan.a[w]
    Mr = state.plan.M[w] // 2 + 1
    buf = np.zeros((N, Mr, 2), np.float32)
    _check(lib().mp_state_coefficients(state.handle, sig, w, buf.ctypes.data, buf.size))
    return buf[..., 0] + 1j * buf[..., 1]


def _status_arrays(B):
    return np.zeros(B, np.int64), np.zeros(B, np.int32), np.zeros(B, np.float64)


def mp_run(state: State, K_max: int, target_snr_db: float, allow_timeout=False):
    """Returns (n_atoms[B], stop_reason[B], snr_db[B]); raises on error.
    With allow_timeout, MP_ETIMEOUT is returned as a flag instead."""
    n, s, q = _status_arrays(state.B)
    rc = lib().mp_run(state.handle, int(K_max), float(target_snr_db), n.ctypes.data, s.ctypes.data,
                      q.ctypes.data)
    if allow_timeout and rc == MP_ETIMEOUT:
        return n, s, q, True
    _check(rc)
    return (n, s, q, False) if allow_timeout else (n, s, q)


def mp_run_async(state: State, K_max: int, target_snr_db: float):
    _check(lib().mp_run_async(state.handle, int(K_max), float(target_snr_db)))


def mp_get_status(state: State):
    n, s, q = _status_arrays(state.B)
    _check(lib().mp_get_status(state.handle, n.ctypes.data, s.ctypes.data, q.ctypes.data))
    return n, s, q


def mp_state_set_time_limit(state: State, seconds: float):
    _check(lib().mp_state_set_time_limit(state.handle, float(seconds)))


def mp_state_set_launch(state: State, threads: int = 0, cluster: int = 0):
    """Pin the MP launch shape (threads per CTA, CTAs per signal); 0, 0
    restores the default."""
    _check(lib().mp_state_set_launch(state.handle, int(threads), int(cluster)))


def mp_state_get_launch(state: State):
    t, c = C.c_int(), C.c_int()
    _check(lib().mp_state_get_launch(state.handle, C.byref(t), C.byref(c)))
    return t.value, c.value


def mp_state_set_top_keys(state: State, max_keys: int = 0):
    """Cap the on-chip top level of a one-CTA-per-signal launch at max_keys
    keys (a power of two; frames are grouped to fit); 0 restores the
    default."""
    _check(lib().mp_state_set_top_keys(state.handle, int(max_keys)))


def mp_state_get_top_keys(state: State) -> int:
    k = C.c_int()
    _check(lib().mp_state_get_top_keys(state.handle, C.byref(k)))
    return k.value


def mp_state_set_work_hint(state: State, work=None):
    """Start the signals with the most work first (work: B non-negative
    numbers, e.g. atoms needed in an earlier run); None: longest first."""
    if work is None:
        _check(lib().mp_state_set_work_hint(state.handle, None))
        return
    w = np.ascontiguousarray(work, dtype=np.float64)
    if w.shape != (state.B,):
        raise ValueError("work needs one entry per signal")
    _check(lib().mp_state_set_work_hint(state.handle, w.ctypes.data))


def mp_state_set_resets(state: State, reset_every: int = 0, reset_err_db: float = 0.0):
    """Alg. 2 resets: after reset_every selections since the last reset, or
    once 10 log10(E_k / E_out) < reset_err_db (< 0); 0 disables either."""
    _check(lib().mp_state_set_resets(state.handle, int(reset_every), float(reset_err_db)))


def mp_get_atoms(state: State, sig: int, cap: int | None = None):
    n = C.c_int64()
    _check(lib().mp_get_atoms(state.handle, sig, None, 0, C.byref(n)))
    k = n.value if cap is None else min(n.value, cap)
    out = np.zeros(k, ATOM_DTYPE)
    if k:
        _check(lib().mp_get_atoms(state.handle, sig, out.ctypes.data, k, C.byref(n)))
    return out


def mp_get_errors(state: State, sig: int):
    n = C.c_int64()
    _check(lib().mp_get_errors(state.handle, sig, None, 0, C.byref(n)))
    out = np.zeros(n.value, np.float64)
    if n.value:
        _check(lib().mp_get_errors(state.handle, sig, out.ctypes.data, n.value, C.byref(n)))
    return out


def mp_synthesize(state: State, sig: int, y, want_snr: bool = True):
    """Writes the approximation of signal `sig` into the float32 CUDA tensor y;
    returns the true residual SNR in dB (or None)."""
    if not (y.is_cuda and y.numel() == state.L[sig] and str(y.dtype) == "torch.float32"):
        raise ValueError("y must be a float32 CUDA tensor of the signal's length")
    snr = C.c_double()
    _check(lib().mp_synthesize(state.handle, sig, y.data_ptr(), C.byref(snr) if want_snr else None))
    return snr.value if want_snr else None


def mp_state_destroy(state: State):
    state.close()


def mp_last_error() -> str:
    return lib().mp_last_error().decode(errors="replace")


def mp_decompose_static(plan: Plan, x, K_max: int, target_snr_db: float, atoms_out,
                        errors_out=None, sync=True):
    """Allocation-free analysis + MP of one signal (see include/mpgabor.h).

    x: float32 CUDA tensor; atoms_out: CUDA tensor of at least K_max * 24
    bytes (e.g. torch.empty(K_max * 24, dtype=torch.uint8)); errors_out:
    float64 CUDA tensor of K_max entries or None.  The plan's stream is
    ordered after torch's current stream before the call (inputs written
    there are ready) and torch's current stream after the plan's stream
    afterwards (the outputs are ready for work queued there).
    sync=True: returns (n_atoms, stop, snr_db) after synchronising the
    plan's stream.  sync=False: passes no host outputs, so the call only
    enqueues its work and returns None; atoms_out then holds the atoms in
    order, and unused entries keep their previous contents.  The atoms are
    read back with atoms_from_bytes()."""
    if not (x.is_cuda and x.is_contiguous() and str(x.dtype) == "torch.float32"):
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    if atoms_out.numel() * atoms_out.element_size() < int(K_max) * ATOM_DTYPE.itemsize:
        raise ValueError("atoms_out is too small")
    if errors_out is not None and errors_out.numel() < int(K_max):
        raise ValueError("errors_out is too small")
    n, s, q = C.c_int64(), C.c_int(), C.c_double()
    outs = (C.byref(n), C.byref(s), C.byref(q)) if sync else (None, None, None)
    _wait_for_current(plan)
    _check(lib().mp_decompose_static(plan.handle, x.data_ptr(), int(x.numel()), int(K_max),
                                     float(target_snr_db), atoms_out.data_ptr(),
                                     errors_out.data_ptr() if errors_out is not None else None,
                                     *outs))
    _current_waits_for_plan(plan)
    return (n.value, s.value, q.value) if sync else None


def atoms_from_bytes(buf, n):
    """View the first n records of a byte buffer (numpy) as mp_atom."""
    return np.frombuffer(np.ascontiguousarray(buf).tobytes(), dtype=ATOM_DTYPE, count=int(n))

"""Host-side helpers of bench.py (CPU): the oracle comparison it reports and
the code hash that guards the profiled DRAM figures."""
import os

import numpy as np

import bench
from oracle import cmp
from paper_2202_12380_gb300 import inputs

ATOM = np.dtype([("dict", "<i4"), ("m", "<i4"), ("n", "<i8"), ("re", "<f4"), ("im", "<f4")])


def _ref():
    dicts = [(inputs.blackman(64), 16, 64), (inputs.blackman(128), 32, 128)]
    return cmp.mp_coef(dicts, inputs.mixture(2048, 82, fs=8000.0), 1e-4, 200, 200.0)


def _as_gpu(ref):
    a = np.zeros(ref.n_atoms, ATOM)
    a["dict"], a["m"], a["n"] = ref.dict, ref.m, ref.n
    a["re"], a["im"] = ref.c.real, ref.c.imag
    return a


def test_oracle_error_of_identical_decomposition():
    ref = _ref()
    r = bench.oracle_error(_as_gpu(ref), ref.E.copy(), ref.E0, ref)
    assert r["first_divergence"] == ref.n_atoms
    assert r["compared"] == r["first_near_tie"] <= ref.n_atoms
    assert r["coef_rel_max"] < 1e-6 and r["snr_db_max_common"] < 1e-9


def test_oracle_error_sees_a_divergence():
    ref = _ref()
    a = _as_gpu(ref)
    a["m"][30] += 1
    r = bench.oracle_error(a, ref.E.copy(), ref.E0, ref)
    assert r["first_divergence"] == 30 and r["compared"] <= 30


def test_code_hash_ignores_comments_only(tmp_path):
    src = "int f(int x) {  // doubles\n    return 2 * x;\n}\n"
    p1, p2, p3 = (os.path.join(tmp_path, n) for n in ("a.cu", "b.cu", "c.cu"))
    open(p1, "w").write(src)
    open(p2, "w").write("// header\n\n" + src.replace("// doubles", "// twice"))
    open(p3, "w").write(src.replace("2 * x", "3 * x"))
    assert bench.code_sha256(p1) == bench.code_sha256(p2)
    assert bench.code_sha256(p1) != bench.code_sha256(p3)


def test_batched_cpu_baseline_uses_a_process_pool():
    r = bench.cpu_baseline_batched(every=128, workers=2)
    assert r["kind"] == "oracle" and r["cores"] == 2 and r["value"] > 0
    assert "2 of the 256 batch256 signals" in r["sample"]
    assert r["host"]["nproc"] >= 1


def test_stored_oracle_prefix_matches_this_host_input():
    import hashlib
    ref = bench._stored_oracle_prefix("multi5_2p20")
    assert ref is not None and ref.n_atoms == 2000
    x = inputs.workload_signal("multi5_2p20")
    assert hashlib.sha256(np.ascontiguousarray(x, np.float32).tobytes()).hexdigest() == \
        ref.input_sha256

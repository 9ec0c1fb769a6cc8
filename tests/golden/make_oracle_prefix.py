"""Writes the FP64 oracle's first atoms of a workload to a golden file.

The bench reports the error of a GPU decomposition of the multi5_2p20
workload (L = 2^20, five Blackman dictionaries) against the oracle, whose
analysis of that signal alone takes tens of seconds on one host core; the
stored prefix written here (by the oracle only) stands in for a live run.
The file records the sha256 of the float32 input so that a host whose input
generator produced other samples is detected.

    python tests/golden/make_oracle_prefix.py multi5_2p20 2000
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import cmp  # noqa: E402
from paper_2202_12380_gb300 import inputs  # noqa: E402


def input_sha256(x):
    return hashlib.sha256(np.ascontiguousarray(x, np.float32).tobytes()).hexdigest()


def main(name, K):
    cfg = inputs.WORKLOADS[name]
    dicts = [(inputs.make_window(k, w), a, M) for (k, w, a, M) in cfg["dicts"]]
    x = inputs.workload_signal(name)
    ref = cmp.mp_coef(dicts, x.astype(np.float64), cfg["eps"], K, cfg["snr_db"])
    out = os.path.join(HERE, "%s_oracle_prefix.npz" % name)
    np.savez_compressed(out, dict=ref.dict, m=ref.m, n=ref.n, c=ref.c, E=ref.E, s1=ref.s1,
                        s2=ref.s2, E0=np.float64(ref.E0), stop=np.int32(ref.stop),
                        input_sha256=np.array(input_sha256(x)), K=np.int64(K))
    print(out, ref.n_atoms, "atoms")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "multi5_2p20",
         int(sys.argv[2]) if len(sys.argv) > 2 else 2000)

"""FP64 CPU oracle for multi-Gabor matching pursuit.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
bench's cpu_baseline / reference legs, never by the product path.  It shares
no code with the CUDA library; the two meet only through the seeded input
generators in ``paper_2202_12380_gb300.inputs``.

* ``oracle.cmp``      -- ctypes front end of the C oracle (mp_oracle.c):
                         kernels, DGT, coefficient-domain MP (Alg. 1 + 3),
                         plain signal-domain MP, synthesis.
* ``oracle.explicit`` -- numpy oracle with an explicit dictionary matrix D
                         (eq. gabdict) for tiny signals: Gram matrix D^* D and
                         MP by its definition with least-squares real pairs.
"""

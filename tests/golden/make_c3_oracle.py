"""Writes c3_oracle_4096x2048.npz: the CPU oracle's SVD (Alg. zvjsvd, FP64)
of the complex 4096 x 2048 workload A = Q1 diag(s) Q2^H (s geometric from 1
down to 1e-6), for the full-size GPU tests and the benchmark to state their
error against the oracle per output.

Stored: all 2048 singular values (as doubles and as the (e, f) pair), the
columns COLS of U and V, the oracle's sweep and rotation counts, and a hash
of the input so that a reader can tell whether its own input is bit-equal
to this one (the generator's QR goes through LAPACK, whose last bits may
differ between machines; such a difference moves the SVD far less than the
tolerances the readers apply).

Calls only the seeded input generator and oracle/; it takes about two hours
on eight cores.  Run from the repository root:
    python tests/golden/make_c3_oracle.py [threads]
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2202_08361_gb300 import workloads  # noqa: E402

COLS = np.array([0, 1, 512, 1023, 1024, 1535, 2046, 2047])
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle_4096x2048.npz")


def input_hash(A):
    return hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else 0
    A, s = workloads.svd_complex_geometric()
    h = input_hash(A)
    t0 = time.time()
    r = oracle.vjsvd(A, nthreads=threads)
    dt = time.time() - t0
    assert r["status"] == oracle.OK, r["status"]
    np.savez(OUT, sigma=r["sigma"], sigma_e=r["sigma_e"], sigma_f=r["sigma_f"], cols=COLS,
             U_cols=np.ascontiguousarray(r["U"][:, COLS]),
             V_cols=np.ascontiguousarray(r["V"][:, COLS]),
             sweeps=r["sweeps"], rotations=r["rotations"], input_sha256=h,
             seconds=dt, threads=oracle.num_threads())
    print("wrote", OUT, "sweeps", r["sweeps"], "seconds", round(dt, 1))


if __name__ == "__main__":
    main()

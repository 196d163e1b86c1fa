"""Build the CPU oracle (test infrastructure only) into oracle/_build/.

The oracle is plain C compiled with -ffp-contract=off so that no multiply
and add are fused behind the source's back: every fused multiply-add in the
oracle is an explicit fma() call, as in the paper's listings.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "jsvd_oracle.c")
SRC_Q = os.path.join(HERE, "jsvd_oracle_q.c")  # the binary128 twin
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libjsvd_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(SRC_Q))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-fvisibility=hidden",
           "-Wall", "-Wextra", "-o", tmp, SRC, SRC_Q, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def build_mutant(k: int, out_dir: str) -> str:
    """The oracle with planted mistake number k (ORC_MUTANT = k, see MUT in
    jsvd_oracle.c) in out_dir, for the tests that check the pins catch it."""
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libjsvd_oracle_m%d.so" % k)
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-fvisibility=hidden",
           "-DORC_MUTANT=%d" % k, "-o", lib, SRC, SRC_Q, "-lm"]
    subprocess.run(cmd, check=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

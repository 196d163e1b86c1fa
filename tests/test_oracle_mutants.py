"""The pins catch plausible mistakes in the oracle.  Each case builds the
oracle with one planted mistake (ORC_MUTANT = k: a dropped term, a wrong
sign or index, a transposed operand, a missing square root) and runs the
pins meant to catch it, in a subprocess loading that library; they must
fail.  A control run of the same pins on the plain oracle must pass."""
import os
import subprocess
import sys

import pytest

from oracle import build as oracle_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# mutant: (what is planted, the pins that must catch it)
MUTANTS = {
    1: ("lambda1' takes a11 where Eq. e:lamsec has a22",
        "tests/test_oracle_evd.py::test_eigenvalues_closed_form"),
    2: ("cos(phi) = 1/sec^2 instead of 1/sec",
        "tests/test_oracle_evd.py::test_prop_2_1_rotation_bounds"),
    3: ("tan(phi) without the sign of a21 (Alg. d8jac2)",
        "tests/test_oracle_evd.py::test_residual_and_orientation"),
    4: ("sin(alpha) with the wrong sign (Eq. e:zpolar)",
        "tests/test_oracle_evd.py::test_residual_and_orientation"),
    5: ("eta off by one in Eq. e:z",
        "tests/test_oracle_evd.py::test_scaling_exponent_cases"),
    6: ("the conjugate on the wrong column of g_q^* g_p (Alg. zdpscl)",
        "tests/test_oracle_svd.py::test_svd_complex_geometric"),
    7: ("a wrong sign in the rotation of Eq. e:transf",
        "tests/test_oracle_svd.py::test_svd_real_geometric"),
    8: ("a wrong index in the round-robin ordering",
        "tests/test_oracle_svd.py::test_pairs_round_robin"),
    9: ("no doubling of f for an odd exponent in the (e, f) square root (SM6.1)",
        "tests/test_oracle_rnf.py"),
    10: ("the carried error t dropped from the compensated sum (Alg. zdpscl')",
         "tests/test_oracle_compensated.py"),
    11: ("psi with the wrong sign in Eq. e:GS",
          "tests/test_oracle_svd.py::test_gram_schmidt_branch"),
    12: ("F_ij = 1/(s_i^2 - s_j^2) swapped in the adjoint",
          "tests/test_oracle_svd.py::test_adjoint_central_differences"),
    13: ("binary32 cos(phi) = 1/sec^2",
          "tests/test_oracle_evd_fp32.py::test_prop_2_1_rotation_bounds"),
    14: ("fma(fh, fr, fr) in the (e, f) step of SM6.2",
          "tests/test_oracle_rnf.py"),
    15: ("the scaled Grammian's a22 built from f_p/f_q (Alg. Gram)",
          "tests/test_oracle_svd.py::test_svd_real_geometric"),
    16: ("tan(phi) = tan(2phi) / (2 + sqrt(...)) in the binary128 twin",
          "tests/test_oracle_twin.py::test_twin_evd_against_exact"),
    17: ("the compensated imaginary stream with the wrong sign (reading R19)",
          "tests/test_oracle_compensated.py"),
    18: ("the rescaling of section 3.2 without its update s += s_[k]",
          "tests/test_oracle_svd.py::test_rescale_branch_is_exact"),
    19: ("the rescaling of section 3.2 scales G by 2^-s_[k] (wrong sign)",
          "tests/test_oracle_svd.py::test_rescale_branch_is_exact"),
}


def _run_pins(lib, pins):
    env = dict(os.environ, ORC_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"]
    cmd += pins.split()
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_control_plain_oracle_passes_the_pins(tmp_path):
    lib = oracle_build.build_mutant(0, str(tmp_path))
    pins = " ".join(sorted({p for _, p in MUTANTS.values()}))
    r = _run_pins(lib, pins)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_catch_planted_mistake(k, tmp_path):
    what, pins = MUTANTS[k]
    lib = oracle_build.build_mutant(k, str(tmp_path))
    r = _run_pins(lib, pins)
    assert r.returncode != 0, "mutant %d (%s) passed %s" % (k, what, pins)
    assert "failed" in r.stdout or "Error" in r.stdout, r.stdout[-2000:]

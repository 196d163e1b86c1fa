"""The integer-pipe binary64 division and square root (csrc/fp64soft.cuh, fp64sel.cuh),
and their select-based forms with the exact x 2^k (also its fast path for
warp-uniform operands) and the scaled comparison of Eq. e:GScond, bit for
bit against IEEE
arithmetic: on the host against the CPU's
correctly rounded division and square root, on the GPU against the FP64
pipe's instructions; and the 2x2 EVD with every division placement."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_against_ieee(tmp_path):
    exe = str(tmp_path / "soft_fp64_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                    "-I" + os.path.join(ROOT, "paper_2202_08361_gb300", "csrc"), "-o", exe,
                    os.path.join(ROOT, "tests", "native", "soft_fp64_check.cpp")], check=True)
    for seed in (1, 2):
        out = subprocess.run([exe, "3000000", str(seed)], check=True, capture_output=True,
                             text=True).stdout.split()
        assert out == ["0"] * 7, out


@pytest.mark.gpu
def test_device_against_fp64_pipe():
    import torch
    from paper_2202_08361_gb300 import _native
    bad = torch.zeros(2, dtype=torch.int64, device="cuda")
    for seed in (0, 1 << 40):
        rc = _native.lib().jsvd_selftest_fp64(1 << 29, seed, bad.data_ptr(), None)
        assert rc == 0
    torch.cuda.synchronize()
    assert bad.tolist() == [0, 0]


def _check_evd_against_oracle(J, salt, tag):
    import torch
    import oracle
    from paper_2202_08361_gb300 import workloads
    for cplx in (False, True):
        streams = workloads.evd_batch(1 << 18, cplx, seed_salt=salt)
        t = [torch.from_numpy(a).cuda() for a in streams]
        out = J.evd2x2_batched(t[0], t[1], t[2], t[3] if cplx else None)
        ref = oracle.zsjac2(*streams) if cplx else oracle.dsjac2(*streams)
        keys = (["cos_phi", "ea_tan_re", "ea_tan_im", "lambda1", "lambda2", "zeta_p"] if cplx
                else ["cos_phi", "ea_tan_re", "lambda1", "lambda2", "zeta_p"])
        for k, r in zip(keys, ref):
            g = out[k].cpu().numpy()
            assert np.array_equal(g.view(np.uint8), np.asarray(r).view(np.uint8)), (tag, cplx, k)


@pytest.mark.gpu
@pytest.mark.parametrize("variant", range(8))
def test_evd_division_placements_bit_identical(variant):
    """Every placement of the EVD's divisions and roots gives the oracle's
    bits (the placement is a launch knob, not an arithmetic choice)."""
    import paper_2202_08361_gb300 as J
    try:
        J.tune_set(J.JSVD_TUNE_EVD_ARITH, variant)
        _check_evd_against_oracle(J, variant, variant)
    finally:
        J.tune_set(J.JSVD_TUNE_EVD_ARITH, -1)


@pytest.mark.gpu
def test_evd_per_field_placements_bit_identical():
    """Different placements for the real and the complex kernel."""
    import paper_2202_08361_gb300 as J
    try:
        J.tune_set(J.JSVD_TUNE_EVD_ARITH, 7, 1)
        J.tune_set(J.JSVD_TUNE_EVD_ARITH, 1, 2)
        _check_evd_against_oracle(J, 77, "real 7, complex 1")
    finally:
        J.tune_set(J.JSVD_TUNE_EVD_ARITH, -1)

"""Parity of the single precision batched 2x2 EVD (jsvd_evd2x2_batched_f32)
with the oracle's binary32 EVD (Listing 1 / Alg. d8jac2 with the binary32
constants of section 2.4): the same operation sequence in binary32 with
round-to-nearest, so the outputs must agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

KEYS_R = ["cos_phi", "ea_tan_re", "lambda1", "lambda2", "zeta_p"]
KEYS_C = ["cos_phi", "ea_tan_re", "ea_tan_im", "lambda1", "lambda2", "zeta_p"]


def run_gpu(streams, complex_):
    import torch
    import paper_2202_08361_gb300 as J
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in streams]
    out = J.evd2x2_batched(t[0], t[1], t[2], t[3] if complex_ else None)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def check(streams, complex_):
    g = run_gpu(streams, complex_)
    ref = oracle.csjac2(*streams) if complex_ else oracle.ssjac2(*streams)
    for k, r in zip(KEYS_C if complex_ else KEYS_R, ref):
        assert g[k].dtype == np.asarray(r).dtype, k
        bad = np.nonzero(g[k].view(np.uint32) != np.asarray(r).view(np.uint32))[0]
        assert bad.size == 0, (k, bad[:5], [s[bad[0]] for s in streams])


@pytest.fixture(params=[0, 1, 2, 4, 7], ids=lambda v: "div_placement_%d" % v)
def div_mode(request):
    """Placements of the single precision EVD's divisions between the IEEE
    and the branch-free routine (JSVD_TUNE_EVD32_DIV): none, all, the
    default, two subsets."""
    import paper_2202_08361_gb300 as J
    J.tune_set(J.JSVD_TUNE_EVD32_DIV, request.param)
    yield request.param
    J.tune_set(J.JSVD_TUNE_EVD32_DIV, -1)


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [1, 7, 1000, 65537, (1 << 20) + 13])
def test_parity_wide_range(n, complex_, div_mode):
    check(workloads.evd_batch_f32(n, complex_, seed_salt=n % 97), complex_)


def test_branch_free_division_against_ieee():
    """The branch-free binary32 division against the IEEE division on 2^30
    operand pairs of every kind (subnormal quotients and operands, overflow,
    zeros, zero divisors)."""
    import torch
    from paper_2202_08361_gb300 import _native
    bad = torch.zeros(1, dtype=torch.int64, device="cuda")
    for seed in (0, 1 << 40):
        assert _native.lib().jsvd_selftest_fp32div(1 << 29, seed, bad.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert bad.item() == 0


@pytest.mark.parametrize("complex_", [False, True])
def test_parity_special_cases(complex_, div_mode):
    fmax = np.finfo(np.float32).max
    tiny = np.float32(2.0 ** -149)
    vals = np.array([0.0, -0.0, 1.0, -1.0, tiny, -tiny, fmax, -fmax, fmax / 8, 2.0 ** -126,
                     3.0, 0.5], dtype=np.float32)
    import itertools
    combos = np.array(list(itertools.product(vals, repeat=4 if complex_ else 3)), dtype=np.float32)
    check(tuple(np.ascontiguousarray(combos[:, k]) for k in range(combos.shape[1])), complex_)


def test_full_size_sample_and_launch_shapes():
    """2^24 matrices (the FP64 workload's size) in every launch shape give the
    same bits; a sample matches the oracle."""
    import torch
    import paper_2202_08361_gb300 as J
    n = 1 << 24
    streams = workloads.evd_batch_f32(n, True)
    t = [torch.from_numpy(a).cuda() for a in streams]
    ref = {k: v.clone() for k, v in J.evd2x2_batched(*t).items()}
    try:
        for block, per_sm in ((64, 4), (128, 16), (256, 2)):
            J.tune_set(J.JSVD_TUNE_EVD_LAUNCH, block, per_sm)
            out = J.evd2x2_batched(*t)
            torch.cuda.synchronize()
            for k in ref:
                assert torch.equal(out[k].view(torch.int32), ref[k].view(torch.int32)), (block, k)
    finally:
        J.tune_set(J.JSVD_TUNE_EVD_LAUNCH, 256, 8)
    idx = np.random.default_rng(1).choice(n, 1 << 16, replace=False)
    sub = [a[idx] for a in streams]
    o = oracle.csjac2(*sub)
    for k, r in zip(KEYS_C, o):
        assert np.array_equal(ref[k].cpu().numpy()[idx].view(np.uint32), np.asarray(r).view(np.uint32)), k


def test_dtype_mixing_rejected():
    import torch
    import paper_2202_08361_gb300 as J
    a = torch.zeros(4, dtype=torch.float32, device="cuda")
    b = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        J.evd2x2_batched(a, b, a)

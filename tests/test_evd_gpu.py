"""Parity of the CUDA batched 2x2 EVD (jsvd_evd2x2_batched) with the oracle.

The kernel evaluates the same binary64 operation sequence as the oracle
(Listing 1 / Alg. d8jac2), so bit-for-bit equality is expected; the
acceptance bounds (4 ulp on eigenvalues, 8 ulp on rotation entries) are
checked as well."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

NU = np.finfo(np.float64).max
MU = 5e-324


def _torch():
    import torch
    return torch


def ordered(x):
    i = np.ascontiguousarray(x, dtype=np.float64).view(np.int64)
    return np.where(i >= 0, i, -(i & 0x7FFFFFFFFFFFFFFF))


def ulp_dist(x, y):
    return np.abs(ordered(x) - ordered(y))


def run_gpu(streams, complex_):
    torch = _torch()
    import paper_2202_08361_gb300 as J
    dev = torch.device("cuda:0")
    t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in streams]
    out = J.evd2x2_batched(t[0], t[1], t[2], t[3] if complex_ else None)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def run_oracle(streams, complex_):
    if complex_:
        c, ct, st, l1, l2, zp = oracle.zsjac2(*streams)
        return dict(cos_phi=c, ea_tan_re=ct, ea_tan_im=st, lambda1=l1, lambda2=l2, zeta_p=zp)
    c, ct, l1, l2, zp = oracle.dsjac2(*streams)
    return dict(cos_phi=c, ea_tan_re=ct, lambda1=l1, lambda2=l2, zeta_p=zp)


def assert_parity(g, o):
    for k in ("cos_phi", "ea_tan_re", "ea_tan_im"):
        if k in o:
            assert ulp_dist(g[k], o[k]).max(initial=0) <= 8, k
    for k in ("lambda1", "lambda2"):
        gi, oi = g[k], o[k]
        inf = np.isinf(oi)
        assert np.array_equal(np.isinf(gi), inf) and np.array_equal(gi[inf], oi[inf]), k
        assert ulp_dist(gi[~inf], oi[~inf]).max(initial=0) <= 4, k
    assert np.array_equal(g["zeta_p"], o["zeta_p"])
    # expected: the identical operation sequence gives identical bits
    for k in o:
        assert np.array_equal(np.asarray(g[k]).view(np.uint8), np.asarray(o[k]).view(np.uint8)), k


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [1, 7, 255, 1000, 65537, (1 << 20) + 13])
def test_parity_wide_range(n, complex_):
    streams = workloads.evd_batch(n, complex_, seed_salt=n % 97)
    assert_parity(run_gpu(streams, complex_), run_oracle(streams, complex_))


@pytest.mark.parametrize("complex_", [False, True])
def test_parity_full_size(complex_):
    """The benchmark's batch size (2^24), in the benchmark's launch shape,
    every output compared."""
    streams = workloads.evd_batch(1 << 24, complex_)
    assert_parity(run_gpu(streams, complex_), run_oracle(streams, complex_))


@pytest.mark.parametrize("complex_", [False, True])
def test_parity_prescribed_eigenvalues(complex_):
    streams = workloads.evd_prescribed(1 << 16, complex_)
    assert_parity(run_gpu(streams, complex_), run_oracle(streams, complex_))


def special_cases():
    rows = [
        (NU / 8, NU / 8, MU, MU),      # Eq. e:evil
        (NU / 8, NU / 8, MU, -MU),
        (0.0, 0.0, 0.0, 0.0),          # all zero
        (-0.0, 0.0, -0.0, -0.0),
        (1.0, 1.0, 0.5, 0.0),          # equal diagonal
        (3.0, -2.0, 0.0, 0.0),         # diagonal
        (NU, -NU, NU, NU),             # everything at the top of the range
        (MU, MU, MU, MU),              # everything subnormal
        (MU, 2 * MU, 3 * MU, -MU),
        (1e-310, 1e300, 2e-320, 0.0),  # wide spread
        (1.0, 1.0 + 2**-52, 1e-300, 1e-300),
        (-5.0, 7.0, -0.0, 3.0),
        (2.0**1023, 2.0**-1074, 2.0**-1000, 2.0**1000),
    ]
    cols = list(zip(*rows))
    return [np.array(c) for c in cols]


@pytest.mark.parametrize("complex_", [False, True])
def test_parity_special_cases(complex_):
    a11, a22, ar, ai = special_cases()
    streams = (a11, a22, ar, ai) if complex_ else (a11, a22, ar)
    g = run_gpu(streams, complex_)
    assert_parity(g, run_oracle(streams, complex_))
    if complex_:
        assert g["ea_tan_re"][0] == 1.0 and g["ea_tan_im"][0] == 1.0
        assert g["cos_phi"][0] == 1.0 / np.sqrt(2.0)


def same_bits(x, y):
    torch = _torch()
    if x.dtype == torch.float64:
        x, y = x.view(torch.int64), y.view(torch.int64)
    return torch.equal(x, y)


def test_subranges_and_launch_shapes_bit_identical():
    """Results depend neither on the batch size, the sub-range nor the
    launch shape."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    n = 300001
    a11, a22, ar, ai = (torch.from_numpy(x).cuda() for x in workloads.evd_batch(n, True, 5))
    ref = J.evd2x2_batched(a11, a22, ar, ai)
    try:
        for block, per_sm in ((64, 1), (128, 3), (256, 32)):
            J.tune_set(J.JSVD_TUNE_EVD_LAUNCH, block, per_sm)
            out = J.evd2x2_batched(a11, a22, ar, ai)
            for k in ref:
                assert same_bits(out[k], ref[k]), (block, per_sm, k)
    finally:
        J.tune_set(J.JSVD_TUNE_EVD_LAUNCH, 256, 8)
    for lo, hi in ((0, 1), (17, 1000), (123456, n)):
        out = J.evd2x2_batched(a11[lo:hi], a22[lo:hi], ar[lo:hi], ai[lo:hi])
        for k in ref:
            assert same_bits(out[k], ref[k][lo:hi]), (lo, hi, k)
    torch.cuda.synchronize()


def test_empty_batch_and_optional_outputs():
    torch = _torch()
    import paper_2202_08361_gb300 as J
    z = torch.empty(0, dtype=torch.float64, device="cuda")
    out = J.evd2x2_batched(z, z, z, z)
    assert all(v.numel() == 0 for v in out.values())
    a11, a22, ar = (torch.from_numpy(x).cuda() for x in workloads.evd_batch(1000, False, 3))
    full = J.evd2x2_batched(a11, a22, ar)
    part = J.evd2x2_batched(a11, a22, ar, want_lambda=False, want_zeta_p=False)
    assert set(part) == {"cos_phi", "ea_tan_re"}
    assert torch.equal(part["cos_phi"], full["cos_phi"])
    assert torch.equal(part["ea_tan_re"], full["ea_tan_re"])


@pytest.mark.parametrize("staged", [0, 1])
@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("n", [5, (1 << 20) + 1, 4 * (1 << 20) + 12345])
def test_host_pipeline_bit_identical(n, complex_, staged):
    """jsvd_evd2x2_batched_host on pinned host streams, the kernel reading
    and writing them in place (JSVD_TUNE_EVD_HOST = 0) or staged in chunks
    of 2^20 in three slots (= 1): the same bits as the device call, across
    chunk boundaries, slot reuse and a ragged last chunk; the oracle agrees
    on a sample."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    streams = workloads.evd_batch(n, complex_, seed_salt=17)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in streams]
    J.tune_set(J.JSVD_TUNE_EVD_HOST, staged)
    try:
        out = J.evd2x2_batched_host(*host[:3], host[3] if complex_ else None)
        torch.cuda.synchronize()
    finally:
        J.tune_set(J.JSVD_TUNE_EVD_HOST, 0)
    ref = run_gpu(streams, complex_)
    for k, v in ref.items():
        assert np.array_equal(out[k].numpy().view(np.uint8), v.view(np.uint8)), k
    idx = np.random.default_rng(3).choice(n, min(n, 4096), replace=False)
    sub = [a[idx] for a in streams]
    o = oracle.zsjac2(*sub) if complex_ else oracle.dsjac2(*sub)
    keys = (["cos_phi", "ea_tan_re", "ea_tan_im", "lambda1", "lambda2", "zeta_p"] if complex_
            else ["cos_phi", "ea_tan_re", "lambda1", "lambda2", "zeta_p"])
    for k, r in zip(keys, o):
        assert np.array_equal(out[k].numpy()[idx].view(np.uint8), np.asarray(r).view(np.uint8)), k


def test_host_pipeline_pageable_and_optional_outputs():
    """Pageable host buffers give the same results (copies serialised);
    lambda and zeta_p may be left out; n = 0 is a no-op."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    streams = workloads.evd_batch(70000, True, seed_salt=18)
    host = [torch.from_numpy(np.ascontiguousarray(a)) for a in streams]
    out = J.evd2x2_batched_host(*host, want_lambda=False, want_zeta_p=False)
    torch.cuda.synchronize()
    assert set(out) == {"cos_phi", "ea_tan_re", "ea_tan_im"}
    ref = run_gpu(streams, True)
    for k in out:
        assert np.array_equal(out[k].numpy(), ref[k]), k
    e = torch.empty(0, dtype=torch.float64)
    assert J.evd2x2_batched_host(e, e, e)["cos_phi"].numel() == 0


def test_host_mixed_pinned_pageable_and_offset_views():
    """Pinned inputs with pageable outputs take the staged path; inputs that
    are views at an offset inside one pinned buffer (and outputs likewise)
    are mapped and take the direct path; both give the device call's bits."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    n = 300001
    streams = workloads.evd_batch(n, True, seed_salt=19)
    ref = run_gpu(streams, True)
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in streams]
    out = {k: torch.empty(n, dtype=torch.float64) for k in ("cos_phi", "ea_tan_re", "ea_tan_im",
                                                            "lambda1", "lambda2")}
    out["zeta_p"] = torch.empty(n, dtype=torch.int32)
    r = J.evd2x2_batched_host(*pinned, out=out)
    torch.cuda.synchronize()
    for k in ref:
        assert np.array_equal(r[k].numpy().view(np.uint8), ref[k].view(np.uint8)), k
    big = torch.empty(4 * n + 7, dtype=torch.float64).pin_memory()
    views = [big[3 + j * n: 3 + (j + 1) * n] for j in range(4)]
    for v, a in zip(views, streams):
        v.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    obig = torch.empty(5 * n + 1, dtype=torch.float64).pin_memory()
    out2 = {k: obig[1 + j * n: 1 + (j + 1) * n] for j, k in enumerate(("cos_phi", "ea_tan_re",
                                                                       "ea_tan_im", "lambda1",
                                                                       "lambda2"))}
    out2["zeta_p"] = torch.empty(n, dtype=torch.int32).pin_memory()
    r2 = J.evd2x2_batched_host(*views, out=out2)
    torch.cuda.synchronize()
    for k in ref:
        assert np.array_equal(r2[k].numpy().view(np.uint8), ref[k].view(np.uint8)), k

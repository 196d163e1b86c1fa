"""The batched 2x2 EVD at the largest sizes one GPU holds: more than 2^31
matrices in one call, so that element indices and byte offsets pass 2^31
and 2^34.  Inputs are drawn on the device; outputs are compared bit for bit
with the oracle on a sample that includes both sides of index 2^31 and the
last matrix.  Skipped when the device has too little free memory."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

N = (1 << 31) + 4099


def _torch():
    import torch
    return torch


def _sample(n):
    g = np.random.default_rng(5)
    edge = [0, 1, (1 << 31) - 2, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, n - 2, n - 1]
    return np.unique(np.concatenate([edge, g.integers(0, n, 2048)])).astype(np.int64)


def _need(bytes_):
    torch = _torch()
    free, _ = torch.cuda.mem_get_info()
    if free < bytes_ * 1.1:
        pytest.skip("needs %.0f GB of free device memory, %.0f GB free" % (bytes_ / 1e9, free / 1e9))


def test_fp64_real_beyond_2_31_matrices():
    torch = _torch()
    import paper_2202_08361_gb300 as J
    _need(N * 40)
    gen = torch.Generator(device="cuda").manual_seed(11)
    a = [torch.randn(N, dtype=torch.float64, device="cuda", generator=gen) for _ in range(3)]
    out = J.evd2x2_batched(*a, want_lambda=False, want_zeta_p=False)
    torch.cuda.synchronize()
    idx = _sample(N)
    it = torch.from_numpy(idx).cuda()
    sub = [x.index_select(0, it).cpu().numpy() for x in a]
    got = {k: out[k].index_select(0, it).cpu().numpy() for k in ("cos_phi", "ea_tan_re")}
    del a, out
    torch.cuda.empty_cache()
    c, t, _, _, _ = oracle.dsjac2(*sub)
    assert np.array_equal(got["cos_phi"].view(np.uint64), c.view(np.uint64))
    assert np.array_equal(got["ea_tan_re"].view(np.uint64), t.view(np.uint64))


def test_fp32_real_beyond_2_31_matrices_all_outputs():
    torch = _torch()
    import paper_2202_08361_gb300 as J
    _need(N * 32)
    gen = torch.Generator(device="cuda").manual_seed(12)
    a = [torch.randn(N, dtype=torch.float32, device="cuda", generator=gen) for _ in range(3)]
    out = J.evd2x2_batched(*a)
    torch.cuda.synchronize()
    idx = _sample(N)
    it = torch.from_numpy(idx).cuda()
    sub = [x.index_select(0, it).cpu().numpy() for x in a]
    got = {k: v.index_select(0, it).cpu().numpy() for k, v in out.items()}
    del a, out
    torch.cuda.empty_cache()
    ref = oracle.ssjac2(*sub)
    for k, r in zip(("cos_phi", "ea_tan_re", "lambda1", "lambda2", "zeta_p"), ref):
        assert np.array_equal(got[k].view(np.uint32), np.asarray(r).view(np.uint32)), k

"""jsvd_svd_noalloc: the SVD for callers that cannot allocate device memory
while they run (a framework's caching allocator already holds the GPU's
memory, a latency-critical loop cannot take cudaMalloc's implicit
synchronisation, or the memory footprint is fixed at start-up).  It uses a
fixed 16 MiB scratch array inside the library instead of a workspace
argument; the paper has no counterpart.

Its results are compared, through the C ABI, with jsvd_svd's on calls in a
row (each call finds the previous call's contents in the shared scratch):
both run the same kernels on the same inputs and the library's results do
not depend on where the workspace lies, so they must agree bit for bit.  The
device's free memory must not move across a call once the library's device
code is loaded.  The file is collected last; it also passes alone in a fresh
process."""
import ctypes

import numpy as np
import pytest

from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
KEYS = ("U", "V", "sigma", "sigma_e", "sigma_f")


def tol(n):
    return 64 * n * EPS


def _outputs(torch, m, n, dtype):
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    return {"U": J.colmajor_empty(m, n, dtype, "cuda"), "V": J.colmajor_empty(n, n, dtype, "cuda"),
            "sigma": torch.empty(n, dtype=torch.float64, device="cuda"),
            "sigma_e": torch.empty(n, dtype=torch.float64, device="cuda"),
            "sigma_f": torch.empty(n, dtype=torch.float64, device="cuda"),
            "info": torch.zeros(_native.INFO_BYTES, dtype=torch.uint8, device="cuda")}


def noalloc_svd(A, mode="fp64"):
    """jsvd_svd_noalloc called through the C ABI; the caller allocates only
    its inputs and outputs, before the call.  Also returns how much the
    device's free memory dropped across the call."""
    import torch
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    Ac, lda = J.colmajor(At)
    m, n = A.shape
    cplx = np.iscomplexobj(A)
    out = _outputs(torch, m, n, At.dtype)
    opts = J._opts(mode=J._mode(mode))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc = _native.lib().jsvd_svd_noalloc(
        J.JSVD_COMPLEX if cplx else J.JSVD_REAL, ctypes.byref(opts), m, n, Ac.data_ptr(), lda,
        out["U"].data_ptr(), out["U"].stride(1), out["sigma"].data_ptr(),
        out["sigma_e"].data_ptr(), out["sigma_f"].data_ptr(), out["V"].data_ptr(),
        out["V"].stride(1), out["info"].data_ptr(), stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert rc == 0, rc
    res = {k: np.ascontiguousarray(out[k].cpu().numpy()) for k in KEYS}
    res["info"] = J.decode_info(out["info"])
    res["free_drop"] = free_before - free_after
    return res


def workspace_svd(A, mode="fp64"):
    """The existing entry point, jsvd_svd, with a caller-allocated workspace."""
    import torch
    import paper_2202_08361_gb300 as J
    out = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda(), mode=mode)
    torch.cuda.synchronize()
    res = {k: np.ascontiguousarray(out[k].cpu().numpy()) for k in KEYS}
    res["info"] = J.decode_info(out["info"])
    return res


def test_noalloc_matches_jsvd_svd_calls_in_a_row():
    A1 = workloads.svd_normal(256, 128)
    A2, _ = workloads.svd_geometric(96, 64, 1e6, True, np.random.default_rng(64))
    A3, _ = workloads.svd_geometric(200, 120, 1e4, False, np.random.default_rng(65))
    # plain FP64, then a complex call, then the mixed FP32 -> FP64 mode (which
    # uses more of the scratch: the FP32 planes, the GEMM output, the
    # Newton-Schulz buffers) on top of the earlier calls' contents, then the
    # first matrix again
    calls = [(A1, "fp64"), (A2, "fp64"), (A3, "mixed"), (A1, "fp64")]
    got = [noalloc_svd(A, mode) for A, mode in calls]
    ref = [workspace_svd(A, mode) for A, mode in calls]
    for k, ((A, mode), g, r) in enumerate(zip(calls, got, ref)):
        n = A.shape[1]
        assert g["info"]["status"] == 0, (k, g["info"])
        assert g["info"] == r["info"], (k, g["info"], r["info"])
        for key in KEYS:
            assert np.array_equal(g[key].view(np.uint8), r[key].view(np.uint8)), (k, mode, key)
        res = np.linalg.norm(A - (g["U"] * g["sigma"]) @ g["V"].conj().T) / np.linalg.norm(A)
        assert res <= tol(n), (k, res)
        if k > 0:  # the first call may load the library's device code
            assert g["free_drop"] == 0, (k, g["free_drop"])


def test_noalloc_rejects_problems_beyond_the_scratch():
    import torch
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    m = n = 1024  # needs a little over 16 MiB of workspace
    assert J.svd_workspace_size(m, n) > _native.NOALLOC_SCRATCH_BYTES
    buf = torch.empty(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    rc = _native.lib().jsvd_svd_noalloc(J.JSVD_REAL, None, m, n, p, m, p, m, p, None, None, p, n,
                                        None, None)
    assert rc == J.JSVD_E_WORKSPACE
    # the mixed mode needs more: real 1024 x 512 fits in FP64 but not mixed
    m, n = 1024, 512
    assert J.svd_workspace_size(m, n) <= _native.NOALLOC_SCRATCH_BYTES
    assert J.svd_workspace_size(m, n, mode="mixed") > _native.NOALLOC_SCRATCH_BYTES
    opts = J._opts(mode=J.JSVD_MIXED_FP32_FP64)
    rc = _native.lib().jsvd_svd_noalloc(J.JSVD_REAL, ctypes.byref(opts), m, n, p, m, p, m, p,
                                        None, None, p, n, None, None)
    assert rc == J.JSVD_E_WORKSPACE

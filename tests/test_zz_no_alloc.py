"""jsvd_svd_noalloc: the SVD for callers that cannot allocate device memory
while they run (a framework's caching allocator already holds the GPU's
memory, a latency-critical loop cannot take cudaMalloc's implicit
synchronisation, or the memory footprint is fixed at start-up).  It uses a
fixed 16 MiB scratch array inside the library instead of a workspace
argument; the paper has no counterpart.

Its results are checked, through the C ABI, against jsvd_svd's on two calls
in a row (the second call finds the first call's contents in the shared
scratch), within the tolerance of the SVD tests.  The file is collected
last; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


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


def noalloc_svd(A):
    """jsvd_svd_noalloc called through the C ABI; the caller allocates only
    its inputs and outputs."""
    import torch
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    Ac, lda = J.colmajor(At)
    m, n = A.shape
    cplx = np.iscomplexobj(A)
    out = _outputs(torch, m, n, At.dtype)
    rc = _native.lib().jsvd_svd_noalloc(
        J.JSVD_COMPLEX if cplx else J.JSVD_REAL, None, m, n, Ac.data_ptr(), lda,
        out["U"].data_ptr(), out["U"].stride(1), out["sigma"].data_ptr(),
        out["sigma_e"].data_ptr(), out["sigma_f"].data_ptr(), out["V"].data_ptr(),
        out["V"].stride(1), out["info"].data_ptr(),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("U", "V", "sigma", "sigma_e", "sigma_f")}
    res["info"] = J.decode_info(out["info"])
    return res


def workspace_svd(A):
    """The existing entry point, jsvd_svd, with a caller-allocated workspace."""
    import torch
    import paper_2202_08361_gb300 as J
    out = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda())
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("U", "V", "sigma", "sigma_e", "sigma_f")}
    res["info"] = J.decode_info(out["info"])
    return res


def test_noalloc_matches_jsvd_svd_two_calls_in_a_row():
    A1 = workloads.svd_normal(256, 128)
    A2, _ = workloads.svd_geometric(96, 64, 1e6, True, np.random.default_rng(64))
    got = [noalloc_svd(A1), noalloc_svd(A2)]
    ref = [workspace_svd(A1), workspace_svd(A2)]
    for A, g, r in zip((A1, A2), got, ref):
        n = A.shape[1]
        assert g["info"]["status"] == 0 and g["info"]["sweeps"] == r["info"]["sweeps"]
        assert np.abs(g["sigma"] - r["sigma"]).max() <= tol(n) * r["sigma"][0]
        assert np.abs(g["U"] - r["U"]).max() <= tol(n)
        assert np.abs(g["V"] - r["V"]).max() <= tol(n)
        res = np.linalg.norm(A - (g["U"] * g["sigma"]) @ g["V"].conj().T) / np.linalg.norm(A)
        assert res <= tol(n)


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

"""The single precision SVD (jsvd_svd_f32) against the FP64 oracle on the
same (binary32) matrix: ||A - U S V^H||_F / ||A||_F, max|U^H U - I|,
max|V^H V - I| <= 64 n eps32 and every sigma within 64 n eps32 sigma_max of
the oracle's, eps32 = 2^-23; the bits do not depend on the launch shape."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -23


def tol(n):
    return 64 * n * EPS32


def gpu_svd32(A):
    import torch
    import paper_2202_08361_gb300 as J
    out = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda())
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("U", "V", "sigma")}
    res["info"] = J.decode_info(out["info"])
    return res


def check(A):
    m, n = A.shape
    g = gpu_svd32(A)
    assert g["U"].dtype == A.dtype and g["sigma"].dtype == np.float32
    assert g["info"]["status"] == 0, g["info"]
    A64 = A.astype(np.complex128 if np.iscomplexobj(A) else np.float64)
    U, s, V = (x.astype(A64.dtype) for x in (g["U"], g["sigma"], g["V"]))
    s = s.real
    assert np.linalg.norm(A64 - (U * s) @ V.conj().T) / np.linalg.norm(A64) <= tol(n)
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= tol(n)
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= tol(n)
    assert np.all(np.diff(s) <= 0)
    o = oracle.vjsvd(A64)
    assert np.abs(s - o["sigma"]).max() <= tol(n) * o["sigma"][0]
    return g


@pytest.mark.parametrize("m,n", [(256, 128), (33, 17), (100, 64), (130, 70), (7, 1), (1, 1),
                                 (64, 63)])
def test_real(m, n):
    if (m, n) == (256, 128):
        A = workloads.svd_normal(256, 128)
    else:
        A, _ = workloads.svd_geometric(m, n, 1e3, False, np.random.default_rng(m * 31 + n))
    g = check(np.asfortranarray(A.astype(np.float32)))
    assert g["info"]["sweeps"] < 40


@pytest.mark.parametrize("m,n", [(64, 31), (40, 40), (200, 96)])
def test_complex(m, n):
    A, _ = workloads.svd_geometric(m, n, 1e3, True, np.random.default_rng(m + 7 * n))
    check(np.asfortranarray(A.astype(np.complex64)))


def test_launch_shapes_bit_identical():
    import torch
    import paper_2202_08361_gb300 as J
    A = np.asfortranarray(workloads.svd_normal(256, 128).astype(np.float32))
    ref = gpu_svd32(A)
    try:
        for cap, warps in ((1, 1), (7, 2), (0, 8)):
            J.tune_set(J.JSVD_TUNE_SVD_GRID, cap, warps)
            g = gpu_svd32(A)
            for k in ("U", "V", "sigma"):
                assert np.array_equal(g[k].view(np.uint32), ref[k].view(np.uint32)), (cap, k)
    finally:
        J.tune_set(J.JSVD_TUNE_SVD_GRID, 0, 0)


def test_scaled_inputs_and_zero():
    """Power-of-two scalings near both ends of the binary32 range give the
    scaled results; a zero matrix gives zero singular values."""
    A, _ = workloads.svd_geometric(40, 20, 1e2, False, np.random.default_rng(5))
    A = np.asfortranarray(A.astype(np.float32))
    base = gpu_svd32(A)
    for k in (100, -100):
        g = gpu_svd32(np.asfortranarray(np.ldexp(A, k).astype(np.float32)))
        assert np.array_equal(g["sigma"], np.ldexp(base["sigma"], k).astype(np.float32))
        assert np.array_equal(g["U"], base["U"])
    z = gpu_svd32(np.zeros((9, 4), np.float32, order="F"))
    assert np.all(z["sigma"] == 0) and z["info"]["status"] == 0


@pytest.mark.parametrize("cplx", [False, True])
def test_sigma_against_binary128_twin(cplx):
    """The single precision SVD's singular values against the binary128
    twin's on the same binary32 matrix: within 64 n eps32 sigma_max."""
    A, _ = workloads.svd_geometric(96, 40, 1e3, cplx, np.random.default_rng(71 + cplx))
    A = A.astype(np.complex64 if cplx else np.float32)
    g = gpu_svd32(A)
    t = oracle.q_vjsvd(A.astype(np.complex128 if cplx else np.float64))
    assert t["status"] == 0
    sq = t["sigma"][:, 0]
    assert np.abs(g["sigma"].astype(float) - sq).max() <= tol(40) * sq[0]


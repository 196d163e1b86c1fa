"""The mixed FP32 -> FP64 SVD (jsvd_svd with JSVD_MIXED_FP32_FP64) and its
FP64 GEMM (jsvd_dgemm, the DMMA tensor path).

The mixed SVD must meet the same bounds as the FP64 one against the FP64
oracle: ||A - U S V^H||_F/||A||_F, max|U^H U - I|, max|V^H V - I| <= 64 n eps
and singular values within 64 n eps sigma_max."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads
from tests.golden import c3_fixture

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


def tol(n):
    return 64 * n * EPS


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("transA", [False, True])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (64, 64, 16), (65, 130, 17), (130, 65, 100),
                                   (256, 128, 256), (33, 1, 64), (5, 9, 0)])
def test_dgemm_against_torch(M, N, K, transA):
    torch = _torch()
    import paper_2202_08361_gb300 as J
    g = torch.Generator(device="cpu").manual_seed(M * 1000 + N * 10 + K)
    A = torch.randn((K, M) if transA else (M, K), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((K, N), generator=g, dtype=torch.float64).cuda()
    C0 = torch.randn((M, N), generator=g, dtype=torch.float64).cuda()
    opA = A.t() if transA else A
    C = J.colmajor(C0.clone())[0]
    J.dgemm(A, B, transA=transA, alpha=-0.75, beta=1.5, C=C)
    ref = -0.75 * (opA @ B) + 1.5 * C0
    bound = 4 * max(K, 1) * EPS * (opA.abs() @ B.abs() + C0.abs()).max().item() + 1e-300
    assert (C - ref).abs().max().item() <= bound
    C2 = J.dgemm(A, B, transA=transA)
    assert (C2 - opA @ B).abs().max().item() <= bound


@pytest.mark.parametrize("transA", [False, True])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 5, 3), (64, 32, 16), (65, 130, 17), (130, 65, 100),
                                   (256, 128, 256), (33, 1, 64), (5, 9, 0)])
def test_zgemm_3m_against_torch(M, N, K, transA):
    """jsvd_zgemm's 3M form against torch's complex product, within the 3M
    bound K eps (|Ar| + |Ai|)(|Br| + |Bi|) per entry (times a safety 4)."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    g = torch.Generator(device="cpu").manual_seed(M * 1000 + N * 10 + K + 7)
    A = torch.randn((K, M) if transA else (M, K), generator=g, dtype=torch.complex128).cuda()
    B = torch.randn((K, N), generator=g, dtype=torch.complex128).cuda()
    C0 = torch.randn((M, N), generator=g, dtype=torch.complex128).cuda()
    opA = A.conj().t() if transA else A
    C = J.zgemm(A, B, transA=transA, alpha=-0.75, beta=1.5, C=C0)
    ref = -0.75 * (opA @ B) + 1.5 * C0
    l1 = lambda z: z.real.abs() + z.imag.abs()
    bound = 4 * max(K, 1) * EPS * ((l1(opA) @ l1(B)) + l1(C0)).max().item() + 1e-300
    assert (C - ref).abs().max().item() <= bound
    C2 = J.zgemm(A, B, transA=transA)
    assert (C2 - opA @ B).abs().max().item() <= bound


@pytest.mark.parametrize("K,M", [(1, 1), (17, 33), (100, 64), (300, 97), (2048, 256)])
def test_zgemm_hermitian_gram(K, M):
    """herm=True: A^H A from the tiles on and above the diagonal, exactly
    Hermitian with a zero imaginary diagonal, equal to the general product
    where both form the same entries."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    g = torch.Generator(device="cpu").manual_seed(K * 31 + M)
    A = torch.randn((K, M), generator=g, dtype=torch.complex128).cuda()
    H = J.zgemm(A, transA=True, herm=True)
    assert torch.equal(H, H.conj().t())
    assert torch.equal(H.diagonal().imag, torch.zeros(M, dtype=torch.float64, device=H.device))
    full = J.zgemm(A, A, transA=True)
    iu = torch.triu_indices(M, M, offset=1, device=H.device)
    assert torch.equal(H[iu[0], iu[1]], full[iu[0], iu[1]])
    assert torch.equal(H.diagonal().real, full.diagonal().real)
    l1 = A.real.abs() + A.imag.abs()
    bound = 4 * K * EPS * (l1.t() @ l1).max().item()
    assert (H - A.conj().t() @ A).abs().max().item() <= bound


def gpu_svd(A, **kw):
    torch = _torch()
    import paper_2202_08361_gb300 as J
    out = J.svd(torch.from_numpy(np.asfortranarray(A)).cuda(), **kw)
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("U", "V", "sigma", "sigma_e", "sigma_f")}
    res["info"] = J.decode_info(out["info"])
    return res


def check_bounds(A, g, sigma_ref):
    n = A.shape[1]
    U, s, V = g["U"], g["sigma"], g["V"]
    assert g["info"]["status"] == 0, g["info"]
    res = np.linalg.norm(A - (U * s) @ V.conj().T) / np.linalg.norm(A)
    assert res <= tol(n), res
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= tol(n)
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= tol(n)
    assert np.abs(s - sigma_ref).max() <= tol(n) * sigma_ref[0]
    assert np.all(np.diff(s) <= 0)


@pytest.mark.parametrize("m,n", [(256, 128), (100, 64), (64, 63), (9, 2), (1, 1)])
def test_mixed_real_against_oracle(m, n):
    if (m, n) == (256, 128):
        A = workloads.svd_normal(256, 128)
    else:
        A, _ = workloads.svd_geometric(m, n, 1e4, False, np.random.default_rng(m * 31 + n))
    g = gpu_svd(A, mode="mixed")
    check_bounds(A, g, oracle.vjsvd(A)["sigma"])
    if n > 1:
        assert g["info"]["sweeps_fp32"] > 0


@pytest.mark.parametrize("m,n,cond", [(512, 256, 1e6), (65, 33, 1e3), (40, 40, 1e6)])
def test_mixed_complex_against_oracle(m, n, cond):
    A, s = workloads.svd_geometric(m, n, cond, True, np.random.default_rng(m * 13 + n))
    g = gpu_svd(A, mode="mixed")
    check_bounds(A, g, oracle.vjsvd(A)["sigma"])
    assert np.abs(g["sigma"] - s).max() <= tol(n) * s[0]


def test_mixed_full_size_complex_4096x2048():
    """The complex 4096 x 2048 workload in mixed mode: the same bounds as the
    FP64 path, checked with torch matmuls on the GPU."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    A, s = workloads.svd_complex_geometric()
    At = torch.from_numpy(A).cuda()
    out = J.svd(At, mode="mixed")
    info = J.decode_info(out["info"])
    assert info["status"] == 0, info
    n = A.shape[1]
    U, V, sg = out["U"], out["V"], out["sigma"]
    I = torch.eye(n, dtype=torch.complex128, device="cuda")
    res = torch.linalg.norm(At - (U * sg) @ V.conj().T) / torch.linalg.norm(At)
    assert res.item() <= tol(n)
    assert (U.conj().T @ U - I).abs().max().item() <= tol(n)
    assert (V.conj().T @ V - I).abs().max().item() <= tol(n)
    assert np.abs(sg.cpu().numpy() - s).max() <= tol(n) * s[0]
    # against the oracle's FP64 SVD of the same matrix (stored by
    # tests/golden/make_c3_oracle.py): sigma normwise within 64 n eps, and
    # the sampled singular vectors within the perturbation bound 64 n eps
    # sigma_1 / gap_j
    fx = c3_fixture.load()
    assert fx is not None, "tests/golden/c3_oracle_4096x2048.npz is missing"
    cols = torch.from_numpy(fx["cols"]).cuda()
    e = c3_fixture.errors(sg.cpu().numpy(), U[:, cols].cpu().numpy(), V[:, cols].cpu().numpy(), fx)
    assert e["sigma_max_err_normwise"] <= tol(n), e
    for eu, ev, b in zip(e["U_col_err"], e["V_col_err"], e["col_bound_64neps_over_gap"]):
        assert eu <= b and ev <= b, e


def test_mixed_nonfinite_and_zero():
    import paper_2202_08361_gb300 as J
    A = workloads.svd_normal(8, 4, seed_salt=5)
    A[2, 2] = np.nan
    g = gpu_svd(A, mode="mixed")
    assert g["info"]["status"] == J.JSVD_E_NONFINITE
    g = gpu_svd(np.zeros((6, 3)), mode="mixed")
    assert g["info"]["status"] == 0 and np.all(g["sigma"] == 0)

"""The CUDA one-sided Jacobi SVD (jsvd_svd) against the oracle (Alg. zvjsvd)
and the acceptance bounds: ||A - U S V^H||_F / ||A||_F, max|U^H U - I|,
max|V^H V - I| <= 64 n eps, singular values within 64 n eps sigma_max of the
oracle's; bit-identical results across launch shapes and repeated calls."""
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


def gpu_svd(A, **kw):
    torch = _torch()
    import paper_2202_08361_gb300 as J
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    out = J.svd(At, **kw)
    torch.cuda.synchronize()
    info = J.decode_info(out["info"])
    res = {k: out[k].cpu().numpy() for k in ("U", "V", "sigma", "sigma_e", "sigma_f")}
    res["info"] = info
    return res


def check_accuracy(A, r, n):
    U, s, V = r["U"], r["sigma"], r["V"]
    res = np.linalg.norm(A - (U * s) @ V.conj().T) / np.linalg.norm(A)
    assert res <= tol(n), res
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= tol(n)
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= tol(n)
    assert np.all(np.diff(s) <= 0)


def check_parity(A, g, o):
    n = A.shape[1]
    assert g["info"]["status"] == 0 and o["status"] == 0
    check_accuracy(A, g, n)
    assert np.abs(g["sigma"] - o["sigma"]).max() <= tol(n) * o["sigma"][0]
    # (e, f) form consistent with sigma
    assert np.array_equal(np.ldexp(g["sigma_f"], g["sigma_e"].astype(int)), g["sigma"])
    assert np.all((g["sigma_f"] >= 1.0) & (g["sigma_f"] < 2.0))


def test_ordering_matches_oracle():
    import paper_2202_08361_gb300 as J
    for n in (2, 3, 17, 128, 255, 2048):
        assert np.array_equal(J.ordering(n).cpu().numpy(), oracle.pairs(n)), n


@pytest.mark.parametrize("m,n", [(256, 128), (33, 17), (100, 64), (64, 63), (7, 1), (1, 1),
                                 (2, 2), (300, 129), (64, 32), (97, 96)])
def test_parity_real(m, n):
    if (m, n) == (256, 128):
        A = workloads.svd_normal(256, 128)
    else:
        A, _ = workloads.svd_geometric(m, n, 1e4, False, np.random.default_rng(m * 1000 + n))
    check_parity(A, gpu_svd(A), oracle.vjsvd(A))


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m,n", [(96, 48), (33, 17), (130, 70)])
def test_parity_compensated(m, n, cplx):
    """The compensated dot-products (Alg. zdpscl' / ddpscl', supplement
    SM2.2) against the oracle's compensated SVD: the acceptance bounds, the
    same singular values, sweep counts within one."""
    A, _ = workloads.svd_geometric(m, n, 1e6, cplx, workloads.rng(3, 40 + cplx + m))
    g = gpu_svd(A, compensated=True)
    o = oracle.vjsvd(A, compensated=True)
    check_parity(A, g, o)
    assert abs(g["info"]["sweeps"] - o["sweeps"]) <= 1
    # the plain and the compensated GPU runs differ (the option is live)
    p = gpu_svd(A)
    assert not np.array_equal(p["sigma"], g["sigma"]) or p["info"] != g["info"]


@pytest.mark.parametrize("m,n", [(64, 31), (40, 40)])
def test_parity_permute(m, n):
    """The column swap P applied during the sweeps (section 2, Alg. zvjsvd
    as printed), real and complex."""
    for cplx in (False, True):
        A, _ = workloads.svd_geometric(m, n, 1e5, cplx, np.random.default_rng(m + n))
        check_parity(A, gpu_svd(A, permute=True), oracle.vjsvd(A, permute=True))


@pytest.mark.parametrize("m,n,cond", [(48, 24, 1e6), (65, 33, 1e3), (31, 31, 1e6), (20, 7, 1e2),
                                      (512, 256, 1e6)])
def test_parity_complex(m, n, cond):
    A, s = workloads.svd_geometric(m, n, cond, True, np.random.default_rng(m * 77 + n))
    g = gpu_svd(A)
    check_parity(A, g, oracle.vjsvd(A))
    assert np.abs(g["sigma"] - s).max() <= tol(n) * s[0]


def test_full_size_complex_4096x2048():
    """The complex 4096 x 2048 workload (cond 1e6): the acceptance bounds,
    checked on the GPU with torch matmuls (the oracle would take minutes)."""
    torch = _torch()
    import paper_2202_08361_gb300 as J
    A, s = workloads.svd_complex_geometric()
    At = torch.from_numpy(A).cuda()
    out = J.svd(At)
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


def test_zero_matrix_and_zero_column():
    A = np.zeros((12, 5))
    g = gpu_svd(A)
    assert g["info"]["status"] == 0 and np.all(g["sigma"] == 0) and np.all(g["U"] == 0)
    assert np.array_equal(np.abs(g["V"]), np.eye(5))
    A = workloads.svd_normal(10, 4, seed_salt=4)
    A[:, 2] = 0.0
    g = gpu_svd(A)
    assert g["info"]["status"] == 0 and g["sigma"][-1] == 0.0
    assert np.allclose((g["U"] * g["sigma"]) @ g["V"].T, A, atol=1e-14)


def test_nonfinite_and_not_converged():
    A = workloads.svd_normal(8, 4, seed_salt=5)
    A[3, 1] = np.inf
    g = gpu_svd(A)
    import paper_2202_08361_gb300 as J
    assert g["info"]["status"] == J.JSVD_E_NONFINITE and np.all(np.isnan(g["sigma"]))
    A = workloads.svd_normal(32, 16, seed_salt=6)
    g = gpu_svd(A, max_sweeps=1)
    assert g["info"]["status"] == J.JSVD_NOT_CONVERGED and g["info"]["sweeps"] == 1


def test_rescaling_path():
    """A low rescale bound forces the section 3.2 downscaling; the results
    stay accurate and the exponent bookkeeping keeps sigma unscaled."""
    # nearly rank one: the first column of U S grows to ~sqrt(n) times the
    # entries of A, past the bound 2^1 of the scaled iteration matrix
    A = np.ones((40, 20)) + 0.01 * workloads.svd_normal(40, 20, seed_salt=9)
    g = gpu_svd(A, rescale_exp=1)
    assert g["info"]["rescales"] > 0
    check_parity(A, g, oracle.vjsvd(A))


@pytest.mark.parametrize("k", [1000, -1000])
def test_extreme_scaling(k):
    A0 = workloads.svd_normal(24, 12, seed_salt=3)
    g0 = gpu_svd(A0)
    g = gpu_svd(np.ldexp(A0, k))
    assert g["info"]["status"] == 0
    assert np.array_equal(g["sigma_e"] - k, g0["sigma_e"])
    assert np.array_equal(g["sigma_f"], g0["sigma_f"])
    assert np.array_equal(g["U"], g0["U"]) and np.array_equal(g["V"], g0["V"])


def test_bit_identical_across_launch_shapes():
    import paper_2202_08361_gb300 as J
    A, _ = workloads.svd_geometric(96, 70, 1e5, True, np.random.default_rng(3))
    ref = gpu_svd(A)
    try:
        for cap, warps in ((1, 1), (3, 2), (16, 8), (0, 4), (5, 0)):
            J.tune_set(J.JSVD_TUNE_SVD_GRID, cap, warps)
            g = gpu_svd(A)
            for k in ("U", "V", "sigma"):
                assert np.array_equal(np.ascontiguousarray(g[k]).view(np.uint8),
                                      np.ascontiguousarray(ref[k]).view(np.uint8)), (cap, warps, k)
            assert g["info"] == ref["info"]
    finally:
        J.tune_set(J.JSVD_TUNE_SVD_GRID, 0, 0)
    again = gpu_svd(A)
    assert np.array_equal(np.ascontiguousarray(again["U"]).view(np.uint8),
                          np.ascontiguousarray(ref["U"]).view(np.uint8))


def _step_cases():
    g = np.random.default_rng(41)
    from tests.test_oracle_svd import gs_test_matrix
    A1, _ = workloads.svd_geometric(256, 128, 1e6, False, g)        # one-trip rows, real
    A2, _ = workloads.svd_geometric(128, 64, 1e6, True, g)          # one-trip rows, complex
    A3, _ = workloads.svd_geometric(75, 31, 1e3, False, g)          # ragged rows, odd n
    B = g.standard_normal((60, 12))
    A4 = np.asfortranarray(B * np.ldexp(1.0, -60 * np.arange(12)))   # wide-exponent columns
    A5 = gs_test_matrix(True)                                        # Gram-Schmidt steps
    A6 = g.standard_normal((40, 10))
    A6[:, 3] = 0.0                                                   # a zero column
    return [("real256x128", A1, {}), ("cplx128x64", A2, {}), ("ragged", A3, {}),
            ("permute", A3, {"permute": True}), ("compensated", A2, {"compensated": True}),
            ("wide", A4, {}), ("gram_schmidt", A5, {}), ("zero_col", A6, {}),
            ("rescale", A1, {"rescale_exp": 1}), ("mixed", A1, {"mode": "mixed"})]


@pytest.mark.parametrize("case", range(10))
def test_step_forms_bit_identical(case):
    """The five forms of a sweep step (JSVD_TUNE_SVD_STEP: chunks with one
    rotation per lane; each warp alone with the rotation's independent
    divisions and roots spread over its lanes; the same inside one
    thread-block cluster; four warps per pair with the rows in registers;
    two or four warps per pair with the rows streamed) give the same bits,
    on one-trip and ragged columns, odd n, column swaps, compensated sums,
    the wide-exponent fallback, Gram-Schmidt steps, a zero column, forced
    rescaling and the mixed mode's FP32 phase."""
    import paper_2202_08361_gb300 as J
    name, A, kw = _step_cases()[case]
    outs = []
    try:
        for mode in (1, 2, 3, 4, 5):
            J.tune_set(J.JSVD_TUNE_SVD_STEP, mode)
            outs.append(gpu_svd(A, **kw))
    finally:
        J.tune_set(J.JSVD_TUNE_SVD_STEP, 0)
    a = outs[0]
    assert a["info"]["status"] == 0, name
    for b in outs[1:]:
        for k in ("U", "V", "sigma", "sigma_e", "sigma_f"):
            assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                  np.ascontiguousarray(b[k]).view(np.uint8)), (name, k)
        assert a["info"] == b["info"], name


@pytest.mark.parametrize("case", range(10))
def test_skipping_unchanged_pairs_bit_identical(case):
    """Skipping a pivot pair whose columns have not changed since its last
    meeting (JSVD_TUNE_SVD_SKIP) changes no result, in the per-warp, the
    cluster and the streamed multi-warp step forms, on the step-form cases (rescaling and the mixed
    mode's two phases among them)."""
    import paper_2202_08361_gb300 as J
    name, A, kw = _step_cases()[case]
    try:
        for mode in (2, 3, 5):
            J.tune_set(J.JSVD_TUNE_SVD_STEP, mode)
            outs = []
            for skip in (0, 1):
                J.tune_set(J.JSVD_TUNE_SVD_SKIP, skip)
                outs.append(gpu_svd(A, **kw))
            a, b = outs
            assert a["info"]["status"] == 0, name
            for k in ("U", "V", "sigma", "sigma_e", "sigma_f"):
                assert np.array_equal(np.ascontiguousarray(a[k]).view(np.uint8),
                                      np.ascontiguousarray(b[k]).view(np.uint8)), (name, mode, k)
            assert a["info"] == b["info"], name
    finally:
        J.tune_set(J.JSVD_TUNE_SVD_STEP, 0)
        J.tune_set(J.JSVD_TUNE_SVD_SKIP, 1)


def test_argument_errors():
    import ctypes
    torch = _torch()
    import paper_2202_08361_gb300 as J
    from paper_2202_08361_gb300 import _native
    L = _native.lib()
    w = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    a = torch.empty(64, dtype=torch.float64, device="cuda")
    p = a.data_ptr()
    s = torch.empty(8, dtype=torch.float64, device="cuda").data_ptr()
    assert L.jsvd_svd(5, None, 8, 4, p, 8, p, 8, s, None, None, p, 4, w.data_ptr(), w.numel(), None, None) == -1
    assert L.jsvd_svd(0, None, 4, 8, p, 8, p, 8, s, None, None, p, 8, w.data_ptr(), w.numel(), None, None) == -4
    assert L.jsvd_svd(0, None, 8, 4, p, 7, p, 8, s, None, None, p, 4, w.data_ptr(), w.numel(), None, None) == -6
    assert L.jsvd_svd(0, None, 8, 4, p, 8, p, 8, s, None, None, p, 4, w.data_ptr() + 8, w.numel(), None, None) == -14
    assert L.jsvd_svd(0, None, 8, 4, p, 8, p, 8, s, None, None, p, 4, w.data_ptr(), 16, None, None) == J.JSVD_E_WORKSPACE
    bad = _native.Opts()
    bad.permute = 2
    assert L.jsvd_svd(0, ctypes.byref(bad), 8, 4, p, 8, p, 8, s, None, None, p, 4, w.data_ptr(), w.numel(), None, None) == -2
    bad = _native.Opts()
    bad.compensated = 3
    assert L.jsvd_svd(0, ctypes.byref(bad), 8, 4, p, 8, p, 8, s, None, None, p, 4, w.data_ptr(), w.numel(), None, None) == -2


@pytest.mark.parametrize("cplx", [False, True])
def test_gram_schmidt_branch_matches_oracle(cplx):
    """Supplement SM9's 16 x 16 matrix (column norms ~2^1074 apart): the
    GPU takes Gram-Schmidt steps (Eq. e:GS) as the oracle does, converges,
    and its singular values match LAPACK on the two blocks (the small ones
    after projecting off the large block's span); the batched kernel gives
    the same bits."""
    import torch
    import paper_2202_08361_gb300 as J
    from tests.test_oracle_svd import gs_test_matrix
    G = gs_test_matrix(cplx)
    g = gpu_svd(G)
    o = oracle.vjsvd(G)
    assert g["info"]["status"] == 0 and g["info"]["gs_steps"] > 0 and o["gs"] > 0
    s = g["sigma"]
    U, V = g["U"], g["V"]
    Gs = G * 2.0 ** -1023
    assert np.linalg.norm(Gs - (U * np.ldexp(s, -1023)) @ V.conj().T) / np.linalg.norm(Gs) <= tol(16)
    assert np.abs(U.conj().T @ U - np.eye(16)).max() <= tol(16)
    assert np.abs(V.conj().T @ V - np.eye(16)).max() <= tol(16)
    big = np.linalg.svd(Gs[:, :8], compute_uv=False)
    assert np.all(np.abs(np.ldexp(s[:8], -1023) / big - 1) <= tol(16))
    Q, _ = np.linalg.qr(Gs[:, :8])
    T = G[:, 8:]
    small = np.linalg.svd(T - Q @ (Q.conj().T @ T), compute_uv=False)
    assert np.all(np.abs(s[8:] / small - 1) <= 1e-6)
    assert np.all(np.abs(s / o["sigma"] - 1) <= 1e-6)
    B = J.svd_batched([G])
    torch.cuda.synchronize()
    assert np.array_equal(B.matrix(0)[1].cpu().numpy(), s)
    assert J.decode_info(B.info)["gs_steps"] == g["info"]["gs_steps"]

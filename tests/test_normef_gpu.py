"""The GPU wide-exponent column norms (jsvd_colnorm_ef, Alg. rnF) against the
oracle's rnF and exact cases, and the SVD's wide-exponent fallback for
columns whose squares underflow (graded matrices against the oracle and a
closed form)."""
import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
NU = np.finfo(np.float64).max
MU = 5e-324
EPS = np.finfo(np.float64).eps


def gpu_norms(A):
    import torch
    import paper_2202_08361_gb300 as J
    e, f = J.colnorm_ef(torch.from_numpy(np.asfortranarray(A)).cuda())
    torch.cuda.synchronize()
    return e.cpu().numpy(), f.cpu().numpy()


def rel_diff(e1, f1, e2, f2):
    if e1 == -np.inf or e2 == -np.inf:
        return 0.0 if e1 == e2 else np.inf
    return abs(np.ldexp(f1, int(e1 - e2)) / f2 - 1.0)


@pytest.mark.parametrize("cplx", [False, True])
def test_norms_against_oracle(cplx):
    g = np.random.default_rng(2)
    m, n = 300, 24
    A = g.standard_normal((m, n)) * np.exp2(g.integers(-1000, 1000, (m, n)))
    if cplx:
        A = A + 1j * g.standard_normal((m, n)) * np.exp2(g.integers(-1000, 1000, (m, n)))
    A[:, 3] = 0.0
    A[:, 5] = NU
    A[:, 7] = MU
    e, f = gpu_norms(A)
    for j in range(n):
        col = A[:, j]
        x = np.column_stack([col.real, col.imag]).ravel() if cplx else col
        eo, fo = oracle.rnF(x)
        assert rel_diff(e[j], f[j], eo, fo) <= (m + 4) * U, j
        assert e[j] == -np.inf or (1.0 <= f[j] < 2.0 and e[j] == int(e[j]))
    assert e[3] == -np.inf and f[3] == 1.0


@pytest.mark.parametrize("cplx", [False, True])
def test_long_columns_1024_lanes(cplx):
    """Columns longer than 8192 rows take 1024 lanes: against the oracle's
    one-lane rnF (the error bound of a sum of m squares), exact cases, the
    same bits on every call, and exact power-of-two scale invariance; a
    column of 8192 rows and one of 8193 bracket the switch."""
    g = np.random.default_rng(6 + cplx)
    m, n = 20011, 9
    A = g.standard_normal((m, n)) * np.exp2(g.integers(-900, 900, (m, n)))
    if cplx:
        A = A + 1j * g.standard_normal((m, n)) * np.exp2(g.integers(-900, 900, (m, n)))
    A[:, 2] = 0.0
    A[:, 4] = NU
    A[:, 6] = 0.0
    A[m - 1, 6] = -3.0 * MU
    e, f = gpu_norms(A)
    e2, f2 = gpu_norms(A)
    assert np.array_equal(e, e2) and np.array_equal(f, f2)
    for j in range(n):
        col = A[:, j]
        x = np.column_stack([col.real, col.imag]).ravel() if cplx else col
        eo, fo = oracle.rnF(x)
        assert rel_diff(e[j], f[j], eo, fo) <= (2 * m + 4) * U, j
    assert e[2] == -np.inf and f[2] == 1.0
    assert (e[6], f[6]) == (-1073.0, 1.5)
    B = np.ldexp(g.integers(-(1 << 20), 1 << 20, (m, 3)).astype(float), -20)
    e0, f0 = gpu_norms(B)
    e1, f1 = gpu_norms(np.ldexp(B, -1030))
    assert np.array_equal(e1, e0 - 1030) and np.array_equal(f1, f0)
    for rows in (8192, 8193):
        C = g.standard_normal((rows, 2))
        ec, fc = gpu_norms(C)
        for j in range(2):
            eo, fo = oracle.rnF(C[:, j])
            assert rel_diff(ec[j], fc[j], eo, fo) <= (rows + 4) * U


def test_exact_cases_and_scale_invariance():
    A = np.zeros((70, 4))
    A[:, 0] = NU
    A[13, 1] = -3.0 * MU
    A[:, 2] = MU
    A[40, 3] = 0.75
    e, f = gpu_norms(A)
    eo, fo = oracle.rnF(A[:, 0])
    assert rel_diff(e[0], f[0], eo, fo) <= 74 * U
    assert (e[1], f[1]) == (-1073.0, 1.5)     # one entry: exact
    assert (e[3], f[3]) == (-1.0, 1.5)
    g = np.random.default_rng(4)
    B = np.ldexp(g.integers(-(1 << 20), 1 << 20, (64, 6)).astype(float), -20)
    e0, f0 = gpu_norms(B)
    for k in (-1030, -500, 700):
        e1, f1 = gpu_norms(np.ldexp(B, k))
        assert np.array_equal(e1, e0 + k) and np.array_equal(f1, f0), k


@pytest.mark.parametrize("cplx", [False, True])
def test_svd_graded_closed_form(cplx):
    """A = Q diag(2^(-50 j)): sigma_j = 2^(-50 j) down to 2^-750, where the
    squares of the scaled G underflow; the wide-exponent fallback keeps
    every sigma relatively accurate."""
    import torch
    import paper_2202_08361_gb300 as J
    m, n = 40, 16
    Q = workloads.haar(np.random.default_rng(21 + cplx), m, n, cplx)
    d = np.ldexp(1.0, -50 * np.arange(n))
    A = np.asfortranarray(Q * d)
    out = J.svd(torch.from_numpy(A).cuda())
    torch.cuda.synchronize()
    s = out["sigma"].cpu().numpy()
    assert J.decode_info(out["info"])["status"] == 0
    assert np.all(np.abs(s / d - 1) <= 64 * n * EPS), s / d - 1
    U_ = out["U"].cpu().numpy()
    assert np.abs(U_.conj().T @ U_ - np.eye(n)).max() <= 64 * n * EPS


@pytest.mark.parametrize("cplx", [False, True])
def test_svd_graded_against_oracle(cplx):
    """B D with B random and D = diag(2^(-45 j)): every singular value
    relatively close to the oracle's (one-sided Jacobi is relatively
    accurate on column-graded matrices); batched equals single."""
    import torch
    import paper_2202_08361_gb300 as J
    m, n = 50, 18
    g = np.random.default_rng(33 + cplx)
    B = g.standard_normal((m, n)) + (1j * g.standard_normal((m, n)) if cplx else 0)
    A = np.asfortranarray(B * np.ldexp(1.0, -45 * np.arange(n)))
    o = oracle.vjsvd(A)
    out = J.svd(torch.from_numpy(A).cuda())
    bt = J.svd_batched([A])
    torch.cuda.synchronize()
    s = out["sigma"].cpu().numpy()
    assert np.all(np.abs(s / o["sigma"] - 1) <= 1e-11), s / o["sigma"] - 1
    assert torch.equal(bt.matrix(0)[1].contiguous().view(torch.int64),
                       out["sigma"].contiguous().view(torch.int64))


def test_binding_rejects_other_dtypes():
    """jsvd_colnorm_ef is binary64 only: the binding refuses float32,
    complex64 and integer matrices, and host tensors."""
    import torch
    import paper_2202_08361_gb300 as J
    for dt in (torch.float32, torch.complex64, torch.int64):
        with pytest.raises(TypeError):
            J.colnorm_ef(torch.zeros(8, 3, dtype=dt, device="cuda"))
    with pytest.raises(TypeError):
        J.colnorm_ef(torch.zeros(8, 3, dtype=torch.float64))

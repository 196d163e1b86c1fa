"""Pins of the oracle's one-sided Jacobi SVD (Alg. zvjsvd), its parallel
ordering and the SVD adjoint, against invariants, closed forms, the paper's
worked examples, LAPACK (numpy) and finite differences."""
import math
from decimal import Decimal
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads
from tests.exact import D

EPS64 = np.finfo(np.float64).eps  # 2^-52, the acceptance tolerance unit


def tol(n):
    return 64 * n * EPS64


def check_svd(A, r, bound=None):
    m, n = A.shape
    U, s, V = r["U"], r["sigma"], r["V"]
    b = tol(n) if bound is None else bound
    res = np.linalg.norm(A - (U * s) @ V.conj().T) / np.linalg.norm(A)
    assert res <= b, res
    assert np.abs(U.conj().T @ U - np.eye(n)).max() <= b
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= b
    # sum sigma^2 = ||A||_F^2
    fro2 = np.sum(np.abs(A) ** 2)
    assert abs(np.sum(s ** 2) - fro2) <= n * b * fro2
    # non-increasing order
    assert np.all(np.diff(s) <= 0)


def test_pairs_round_robin():
    """The ordering covers every pair once per sweep with n/2 disjoint pairs
    per step, p < q (section 4.1)."""
    for n in [2, 3, 4, 5, 8, 16, 17, 64, 128, 255, 256]:
        tab = oracle.pairs(n)
        nt = n + (n & 1)
        assert tab.shape == (nt - 1, nt // 2, 2)
        seen = set()
        for k in range(nt - 1):
            step = tab[k]
            cols = step.ravel().tolist()
            assert len(set(cols)) == nt  # disjoint, all columns
            for p, q in step:
                assert 0 <= p < q < nt
                seen.add((int(p), int(q)))
        assert len(seen) == nt * (nt - 1) // 2


def test_svd_real_normal_256x128():
    A = workloads.svd_normal(256, 128)
    r = oracle.vjsvd(A)
    assert r["status"] == oracle.OK
    check_svd(A, r)
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(r["sigma"] - s_ref).max() <= tol(128) * s_ref[0]


@pytest.mark.parametrize("m,n", [(64, 32), (33, 17), (40, 40), (7, 1), (9, 2)])
def test_svd_real_geometric(m, n):
    A, s = workloads.svd_geometric(m, n, 1e4, False, np.random.default_rng(m * 100 + n))
    r = oracle.vjsvd(A)
    assert r["status"] == oracle.OK
    check_svd(A, r)
    assert np.abs(r["sigma"] - s).max() <= tol(n) * s[0]


@pytest.mark.parametrize("cplx", [False, True])
def test_svd_with_column_swaps(cplx):
    """The column swap P of section 2 applied during the sweeps."""
    A, s = workloads.svd_geometric(40, 21, 1e5, cplx, np.random.default_rng(21))
    r = oracle.vjsvd(A, permute=True)
    assert r["status"] == oracle.OK
    check_svd(A, r)
    assert np.abs(r["sigma"] - s).max() <= tol(21) * s[0]


@pytest.mark.parametrize("m,n", [(48, 24), (31, 31), (20, 7)])
def test_svd_complex_geometric(m, n):
    A, s = workloads.svd_geometric(m, n, 1e6, True, np.random.default_rng(m * 7 + n))
    r = oracle.vjsvd(A)
    assert r["status"] == oracle.OK
    check_svd(A, r)
    assert np.abs(r["sigma"] - s).max() <= tol(n) * s[0]
    s_ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(r["sigma"] - s_ref).max() <= tol(n) * s_ref[0]


def test_svd_2x2_closed_form():
    """sigma_{1,2} = sqrt((||A||_F^2 +- sqrt(||A||_F^4 - 4 det^2)) / 2)."""
    g = np.random.default_rng(5)
    for _ in range(50):
        A = g.standard_normal((2, 2)) * 10.0 ** g.integers(-5, 5)
        r = oracle.vjsvd(A)
        f2 = sum(D(x) ** 2 for x in A.ravel())
        det = D(A[0, 0]) * D(A[1, 1]) - D(A[0, 1]) * D(A[1, 0])
        disc = (f2 * f2 - 4 * det * det).sqrt()
        s1, s2 = ((f2 + disc) / 2).sqrt(), ((f2 - disc) / 2).sqrt()
        assert abs(D(r["sigma"][0]) - s1) <= D(8 * EPS64) * s1
        assert abs(D(r["sigma"][1]) - s2) <= D(8 * EPS64) * s1


def test_spectrum_example_xi_minus3():
    """Section 5.1: diag(Sigma[xi=-3, n=4]) = [1/8, 1/4, 1/2, 1]; a permuted
    diagonal input is already orthogonal, so the singular values come out
    exactly, sorted non-increasingly."""
    A = np.zeros((6, 4))
    for j, v in enumerate([0.25, 1.0, 0.125, 0.5]):
        A[j + 1, j] = v
    r = oracle.vjsvd(A)
    assert r["sigma"].tolist() == [1.0, 0.5, 0.25, 0.125]
    assert r["rotations"] == 0


def test_ef_examples():
    """Supplement SM6.1: sqrt(12) = (1, fl(sqrt 3)), sqrt(80) = (3, fl(sqrt 1.25)),
    seen as the single singular value of a column of norm sqrt(12), sqrt(80)."""
    r = oracle.vjsvd(np.array([[2.0], [2.0], [2.0]]))
    assert r["sigma_e"][0] == 1.0 and r["sigma_f"][0] == math.sqrt(3.0)
    r = oracle.vjsvd(np.array([[4.0], [8.0]]))
    assert r["sigma_e"][0] == 3.0 and r["sigma_f"][0] == math.sqrt(1.25)


def test_scaling_extremes():
    """Section 3.2 scaling: a matrix near DBL_MAX and one of subnormal-range
    magnitudes give the same relative results as the unscaled one."""
    A = workloads.svd_normal(24, 12, seed_salt=3)
    r0 = oracle.vjsvd(A)
    for k in (1000, -1000):
        Ak = np.ldexp(A, k)
        r = oracle.vjsvd(Ak)
        assert r["status"] == oracle.OK
        # sigma = 2^e f; compare 2^(e-k) f, which never underflows
        sig = np.ldexp(r["sigma_f"], r["sigma_e"].astype(int) - k)
        assert np.allclose(sig, r0["sigma"], rtol=tol(12), atol=0)
        assert np.array_equal(np.ldexp(r["sigma_f"], r["sigma_e"].astype(int)), r["sigma"])


def test_rank_deficient_zero_column():
    A = workloads.svd_normal(10, 4, seed_salt=4)
    A[:, 2] = 0.0
    r = oracle.vjsvd(A)
    assert r["status"] == oracle.OK
    assert r["sigma"][-1] == 0.0 and np.all(r["U"][:, -1] == 0.0)
    assert np.allclose((r["U"] * r["sigma"]) @ r["V"].T, A, atol=1e-14)


def test_nonfinite_and_not_converged():
    A = workloads.svd_normal(8, 4, seed_salt=5)
    A[3, 1] = np.nan
    with pytest.raises(ValueError):
        oracle.vjsvd(A)
    A = workloads.svd_normal(32, 16, seed_salt=6)
    r = oracle.vjsvd(A, max_sweeps=1)
    assert r["status"] == oracle.NOT_CONVERGED and r["sweeps"] == 1


def test_thread_count_independence():
    """Section 4.3.1: the results do not depend on the number of threads."""
    A = workloads.svd_normal(64, 48, seed_salt=7)
    r1 = oracle.vjsvd(A, nthreads=1)
    r4 = oracle.vjsvd(A, nthreads=4)
    for key in ("U", "V", "sigma"):
        assert np.array_equal(r1[key], r4[key])
    assert r1["sweeps"] == r4["sweeps"] and r1["rotations"] == r4["rotations"]


# ---------------------------------------------------------------------------
# the differentiated batched SVD's loss and its adjoint

def loss(A, w, C, k=8):
    r = oracle.vjsvd(A)
    U, V = oracle.sign_gauge(r["U"], r["V"])
    return float(np.dot(w, r["sigma"]) + np.sum(C * U[:, :k])), r


def test_adjoint_central_differences():
    """A12 adjoint vs central differences (h = 1e-6) along random directions."""
    A, w, C = workloads.diff_batch(count=3, m=20, n=10, cond=1e3, k=4)
    g = np.random.default_rng(9)
    for i in range(3):
        L0, r = loss(A[i], w[i], C[i], k=4)
        U, V = oracle.sign_gauge(r["U"], r["V"])
        Ubar = np.zeros_like(U)
        Ubar[:, :4] = C[i]
        Abar = oracle.svd_adjoint(U, r["sigma"], V, Ubar, w[i])
        for _ in range(3):
            Dd = g.standard_normal(A[i].shape)
            h = 1e-6
            lp, _ = loss(A[i] + h * Dd, w[i], C[i], k=4)
            lm, _ = loss(A[i] - h * Dd, w[i], C[i], k=4)
            fd = (lp - lm) / (2 * h)
            an = float(np.sum(Abar * Dd))
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_adjoint_sigma_only_textbook():
    """With Ubar = Vbar = 0: Abar = U diag(sbar) V^T (d sigma_i/dA = u_i v_i^T)."""
    A = workloads.svd_normal(12, 5, seed_salt=8)
    r = oracle.vjsvd(A)
    sbar = np.arange(1.0, 6.0)
    Abar = oracle.svd_adjoint(r["U"], r["sigma"], r["V"], np.zeros((12, 5)), sbar)
    assert np.allclose(Abar, (r["U"] * sbar) @ r["V"].T, atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_graded_columns_relative_accuracy(cplx):
    """A = Q D, Q with orthonormal columns, D = diag(2^(-50 j)): the singular
    values are D's entries (down to 2^-750), and one-sided Jacobi gets each
    to a few eps relatively (its norms never under- or overflow)."""
    m, n = 40, 16
    Q = workloads.haar(np.random.default_rng(21 + cplx), m, n, cplx)
    d = np.ldexp(1.0, -50 * np.arange(n))
    A = np.asfortranarray(Q * d)
    r = oracle.vjsvd(A)
    assert r["status"] == oracle.OK
    assert np.all(np.abs(r["sigma"] / d - 1) <= 64 * n * EPS64)


def gs_test_matrix(cplx=False):
    """Supplement SM9's 16 x 16 matrix (workloads.gram_schmidt_matrix)."""
    return workloads.gram_schmidt_matrix(cplx)


@pytest.mark.parametrize("cplx", [False, True])
def test_gram_schmidt_branch(cplx):
    """Section 3.5.1 / supplement SM9: the norms of the two column groups
    differ by ~2^1074 > 2^eta^ upsilon, so the pairs across them take the
    Gram-Schmidt step (Eq. e:GS) and the method converges.  The large
    singular values are those of the large block; the small ones those of
    the small block projected off the large block's span (both from LAPACK
    on exactly rescaled copies)."""
    G = gs_test_matrix(cplx)
    r = oracle.vjsvd(G)
    assert r["status"] == oracle.OK and r["gs"] > 0
    U, s, V = r["U"], r["sigma"], r["V"]
    Gs = G * 2.0 ** -1023  # exact: a power-of-two scaling of normal numbers
    res = np.linalg.norm(Gs - (U * np.ldexp(s, -1023)) @ V.conj().T) / np.linalg.norm(Gs)
    assert res <= tol(16)
    assert np.abs(U.conj().T @ U - np.eye(16)).max() <= tol(16)
    assert np.abs(V.conj().T @ V - np.eye(16)).max() <= tol(16)
    big = np.linalg.svd(Gs[:, :8], compute_uv=False)
    assert np.all(np.abs(np.ldexp(s[:8], -1023) / big - 1) <= tol(16))
    Q, _ = np.linalg.qr(Gs[:, :8])
    T = G[:, 8:]
    small = np.linalg.svd(T - Q @ (Q.conj().T @ T), compute_uv=False)
    assert np.all(np.abs(s[8:] / small - 1) <= 1e-6)


def test_gram_schmidt_not_taken_for_moderate_ranges():
    """Eq. e:GScond never holds when the column norms differ by less than
    2^eta^ upsilon: an ordinary matrix takes no Gram-Schmidt step."""
    A, _ = workloads.svd_geometric(60, 30, 1e12, False, np.random.default_rng(4))
    assert oracle.vjsvd(A)["gs"] == 0


@pytest.mark.parametrize("cplx", [False, True])
def test_rescale_branch_is_exact(cplx):
    """The per-step rescaling of section 3.2 (steps 2-4: the test of Eq.
    e:skr, the downscaling by 2^{s_[k]} of Eq. e:skn, the running exponent
    s).  Its threshold is lowered (skr_shift) so that the branch runs on a
    matrix whose max-norm grows during the sweeps: nearly parallel columns,
    whose norm Jacobi gathers into one column (growth about sqrt(n)).
    Power-of-two scaling is exact here (no entry comes near the subnormal
    range), so every output must equal, bit for bit, that of the run that
    never rescales; a dropped or wrong-signed exponent update changes sigma
    by a power of two."""
    rng = np.random.default_rng(77 + cplx)
    m, n = 48, 24
    A = np.ones((m, n)) + 0.01 * rng.standard_normal((m, n))
    if cplx:
        A = A * np.exp(0.3j) + 0.01j * rng.standard_normal((m, n))
    ref = oracle.vjsvd(A)
    assert ref["status"] == oracle.OK and ref["rescales"] == 0
    check_svd(A, ref)
    fired = []
    for shift in (4, 8, 12, 40):
        r = oracle.vjsvd(A, skr_shift=shift)
        fired.append(r["rescales"])
        for k in ("sigma", "sigma_e", "sigma_f", "U", "V"):
            assert np.array_equal(np.ascontiguousarray(r[k]).view(np.uint8),
                                  np.ascontiguousarray(ref[k]).view(np.uint8)), (shift, k)
        assert (r["sweeps"], r["rotations"], r["status"]) == (
            ref["sweeps"], ref["rotations"], ref["status"])
    # the branch ran: a few times once the max-norm doubled, and at every
    # step when the threshold lies below the initial max-norm
    assert fired[-1] >= ref["sweeps"] * (n - 1) and max(fired[:-1]) > 0, fired

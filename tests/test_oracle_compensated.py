"""Pins of the oracle's compensated scaled dot-products (Alg. zdpscl' and
ddpscl', supplement SM2.2) and of the SVD that uses them.

With the norms set to (e, f) = (0, 1) the routine returns the dot-product
itself, which is compared with its exact value in rational arithmetic.
Kahan's summation with 2Sum (item K) bounds the error of a stream by
(2u + O(m u^2)) sum |x_i|, u = 2^-53; on sums of one sign that leaves the
final rounding only, while the plain fma sum (Alg. zdpscl) drifts by many
u -- the test shows both, so it tells the two forms apart."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads

U = 2.0 ** -53


def exact_dot(q, p):
    """q^* p exactly (a pair of Fractions) and sum of |products|."""
    cplx = np.iscomplexobj(q) or np.iscomplexobj(p)
    F = lambda x: Fraction(float(x))
    qr, pr = [F(x) for x in np.real(q)], [F(x) for x in np.real(p)]
    qi = [F(x) for x in np.imag(q)] if cplx else [Fraction(0)] * len(qr)
    pi = [F(x) for x in np.imag(p)] if cplx else [Fraction(0)] * len(pr)
    re = sum(a * b + c * d for a, b, c, d in zip(qr, pr, qi, pi))
    im = sum(a * d - c * b for a, b, c, d in zip(qr, pr, qi, pi))
    ab = sum(abs(a * b) + abs(c * d) + abs(a * d) + abs(c * b) for a, b, c, d in zip(qr, pr, qi, pi))
    return re, im, ab


def err(z, re, im):
    z = complex(z)
    return float(abs(Fraction(z.real) - re)) + float(abs(Fraction(z.imag) - im))


def same_sign_case(seed, m=4096):
    g = np.random.default_rng(seed)
    return g.uniform(0.5, 1.0, m), g.uniform(0.5, 1.0, m)


@pytest.mark.parametrize("seed", range(4))
def test_same_sign_sum_is_rounded_once(seed):
    """All products positive: the compensated dot-product is the exact sum
    rounded once (up to O(m u^2))."""
    q, p = same_sign_case(seed)
    re, im, ab = exact_dot(q, p)
    S = float(re)
    assert err(oracle.dpscl(q, p, True), re, im) <= U * S * (1 + 8 * len(q) * U)


def test_plain_sum_drifts():
    """The same cases with the plain fma sum: off by several u S on
    average, so the test above would catch a compensated form that fell
    back to the plain one."""
    rel = []
    for seed in range(4):
        q, p = same_sign_case(seed)
        re, im, _ = exact_dot(q, p)
        rel.append(err(oracle.dpscl(q, p, False), re, im) / (U * float(re)))
    assert np.mean(rel) > 4.0, rel


def ill_conditioned(m, cplx, seed):
    """q, p whose dot-product cancels to the rounding error of a partial
    sum: the last term is minus the rounded sum of the others."""
    g = np.random.default_rng(seed)
    q = g.standard_normal(m) * np.exp2(g.integers(-8, 8, m))
    p = g.standard_normal(m) * np.exp2(g.integers(-8, 8, m))
    if cplx:
        q = q + 1j * g.standard_normal(m)
        p = p + 1j * g.standard_normal(m)
    head = np.vdot(q[:-1], p[:-1])
    q[-1] = 1.0
    p[-1] = -head
    return q, p


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("seed", range(4))
def test_kahan_bound_on_cancellation(cplx, seed):
    """Condition ~1/u: the error stays within the bound of Kahan's
    summation, (2u + O(m u^2)) sum |x_i y_i| per stream plus the final
    roundings."""
    m = 257
    q, p = ill_conditioned(m, cplx, seed)
    re, im, ab = exact_dot(q, p)
    mag = float(abs(re)) + float(abs(im))
    bound = (2 * U + 16 * m * U * U) * 2 * float(ab) + 4 * U * mag
    assert err(oracle.dpscl(q, p, True), re, im) <= bound


@pytest.mark.parametrize("cplx", [False, True])
def test_moderate_condition_accuracy(cplx):
    """Random vectors: both forms agree with the exact value to a few u of
    sum |x_i y_i| (a wrong sign or a dropped term in either stream would
    not)."""
    g = np.random.default_rng(11)
    m = 300
    q, p = g.standard_normal(m), g.standard_normal(m)
    if cplx:
        q = q + 1j * g.standard_normal(m)
        p = p + 1j * g.standard_normal(m)
    re, im, ab = exact_dot(q, p)
    assert err(oracle.dpscl(q, p, True), re, im) <= 8 * U * float(ab)
    assert err(oracle.dpscl(q, p, False), re, im) <= 2 * m * U * float(ab)


@pytest.mark.parametrize("cplx", [False, True])
def test_exact_sums_agree(cplx):
    """Small integers: every product and partial sum is exact, so both forms
    give the exact value."""
    g = np.random.default_rng(5)
    q = g.integers(-20, 20, 40).astype(float)
    p = g.integers(-20, 20, 40).astype(float)
    if cplx:
        q = q + 1j * g.integers(-20, 20, 40)
        p = p + 1j * g.integers(-20, 20, 40)
    re, im, _ = exact_dot(q, p)
    for comp in (False, True):
        z = complex(oracle.dpscl(q, p, comp))
        assert Fraction(z.real) == re and Fraction(z.imag) == im


def test_scaling_by_the_norms():
    """(e, f) scaling: z = dot / (2^(eq+ep) fq fp), the powers of two exact
    and one division at the end."""
    g = np.random.default_rng(8)
    q, p = g.integers(-9, 9, 30).astype(float), g.integers(-9, 9, 30).astype(float)
    d = float(np.dot(q, p))  # exact: small integers
    for comp in (False, True):
        z = oracle.dpscl(q, p, comp, eq=3, fq=1.25, ep=-2, fp=1.5)
        assert z == (d / 2.0) / (1.25 * 1.5)


@pytest.mark.parametrize("cplx", [False, True])
def test_compensated_svd_meets_bounds(cplx):
    """The SVD with Alg. zdpscl' meets the acceptance bounds, agrees with the
    plain one in sigma, and needs at most one sweep more."""
    m, n = 96, 48
    A, _ = workloads.svd_geometric(m, n, 1e6, cplx, workloads.rng(3, 40 + cplx))
    rc = oracle.vjsvd(A, compensated=True)
    rp = oracle.vjsvd(A)
    assert rc["status"] == oracle.OK
    tol = 64 * n * np.finfo(float).eps
    Uc, s, V = rc["U"], rc["sigma"], rc["V"]
    assert np.linalg.norm(A - (Uc * s) @ V.conj().T) / np.linalg.norm(A) <= tol
    assert np.abs(Uc.conj().T @ Uc - np.eye(n)).max() <= tol
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= tol
    assert np.abs(s - rp["sigma"]).max() <= tol * s[0]
    assert rc["sweeps"] <= rp["sweeps"] + 1

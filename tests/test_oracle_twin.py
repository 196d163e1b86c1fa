"""The binary128 twin of the oracle (oracle/jsvd_oracle_q.c): first pinned
to exact arithmetic (the twin's 2x2 EVD against 80-digit closed forms) and
to LAPACK (its SVD), then used to measure the FP64 oracle with 60 more bits
of reference: the EVD within the Prop. p:s2 bounds on wide-range data, the
SVD's singular values and vectors within the acceptance bounds."""
from decimal import Decimal

import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads
from tests.exact import D, rotation_exact

EPS = 2.0 ** -53
EPS_Q = 2.0 ** -113


def hl(x):
    """exact Decimal of a (hi, lo) pair"""
    return D(float(x[0])) + D(float(x[1]))


def test_twin_evd_against_exact():
    g = np.random.default_rng(3)
    r = 200
    e = lambda: g.integers(-200, 200, r)
    a11, a22, a21r, a21i = (np.ldexp(g.standard_normal(r), e()) for _ in range(4))
    c, tr, ti, l1, l2 = oracle.q_zsjac2(a11, a22, a21r, a21i)
    for i in range(r):
        t, cc, ca, sa = rotation_exact(a11[i], a22[i], a21r[i], a21i[i])
        assert abs(hl(c[i]) - cc) <= D(64 * EPS_Q) * cc
        err = ((hl(tr[i]) - ca * t) ** 2 + (hl(ti[i]) - sa * t) ** 2).sqrt()
        assert err <= D(64 * EPS_Q) * abs(t) + D(2.0 ** -1000)


@pytest.mark.parametrize("complex_", [False, True])
def test_fp64_evd_within_prop_bounds_of_twin(complex_):
    """Prop. p:s2 against the twin on the wide-range batch (entries from
    subnormal to near DBL_MAX): relative errors of cos(phi) and of
    e^{i alpha} tan(phi) within 8 / 14 eps (cos) and the tan bound times
    the e^{i alpha} factor; the eigenvalues of larger magnitude to 16 eps."""
    b = workloads.evd_batch(2000, complex_, seed_salt=5)
    if complex_:
        c, ct, st, l1, l2, _ = oracle.zsjac2(*b)
        qc, qtr, qti, ql1, ql2 = oracle.q_zsjac2(*b)
    else:
        c, ct, l1, l2, _ = oracle.dsjac2(*b)
        st = np.zeros_like(c)
        qc, qtr, qti, ql1, ql2 = oracle.q_zsjac2(b[0], b[1], b[2])
    cos_b = (14.000006 if complex_ else 8.000002) * EPS
    tan_b = (11.500004 if complex_ else 5.500001) * EPS
    et_b = (1 + 4.000001 * EPS) * (1 + tan_b) * (1 + EPS) - 1
    for i in range(len(c)):
        rc = hl(qc[i])
        assert abs(D(c[i]) - rc) <= D(cos_b) * rc, i
        rr, ri = hl(qtr[i]), hl(qti[i])
        mag = (rr * rr + ri * ri).sqrt()
        if mag > 0:
            err = ((D(ct[i]) - rr) ** 2 + (D(st[i]) - ri) ** 2).sqrt()
            assert err <= D(et_b) * mag + D(4.9e-324), i


@pytest.mark.parametrize("cplx", [False, True])
def test_twin_svd_against_lapack(cplx):
    A, s = workloads.svd_geometric(40, 20, 1e5, cplx, np.random.default_rng(7 + cplx))
    r = oracle.q_vjsvd(A)
    assert r["status"] == 0
    sq = r["sigma"][:, 0]
    assert np.abs(sq - np.linalg.svd(A, compute_uv=False)).max() <= 64 * 20 * 2 * EPS * sq[0]
    U, V = r["U"], r["V"]
    assert np.linalg.norm(A - (U * sq) @ V.conj().T) / np.linalg.norm(A) <= 64 * EPS


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("shape", [(64, 32), (33, 33), (50, 7)])
def test_fp64_oracle_svd_against_twin(cplx, shape):
    """The FP64 oracle's singular values within 64 n eps sigma_max of the
    twin's; its singular vectors, for values separated by a relative gap
    above 1e-3, parallel to the twin's up to 64 n eps / gap."""
    m, n = shape
    A, _ = workloads.svd_geometric(m, n, 1e8, cplx, np.random.default_rng(m + n + cplx))
    o = oracle.vjsvd(A)
    t = oracle.q_vjsvd(A)
    assert o["status"] == 0 and t["status"] == 0
    s, sq = o["sigma"], t["sigma"][:, 0]
    tol = 64 * n * 2 * EPS
    assert np.abs(s - sq).max() <= tol * sq[0]
    gaps = np.full(n, np.inf)
    rel = np.abs(np.diff(sq)) / sq[:-1]
    gaps[:-1] = np.minimum(gaps[:-1], rel)
    gaps[1:] = np.minimum(gaps[1:], rel)
    for j in range(n):
        if gaps[j] > 1e-3:
            cu = abs(np.vdot(o["U"][:, j], t["U"][:, j]))
            cv = abs(np.vdot(o["V"][:, j], t["V"][:, j]))
            assert cu >= 1 - tol / gaps[j] * sq[0] / sq[j] and cv >= 1 - tol / gaps[j] * sq[0] / sq[j], j


@pytest.mark.parametrize("complex_", [False, True])
def test_fp32_evd_within_prop_bounds_of_twin(complex_):
    """The binary32 EVD (the constants of section 2.4) against the binary128
    twin on binary32 inputs spread over 2^-40 .. 2^40: Prop. p:s2 with
    eps = 2^-24 (the bounds hold for any precision with at least 23
    fraction bits while nothing underflows)."""
    g = np.random.default_rng(29 + complex_)
    r = 1500
    e = lambda: g.integers(-40, 40, r)
    f = lambda: np.float32(np.ldexp(g.standard_normal(r), e()))
    a11, a22, a21r = f(), f(), f()
    a21i = f() if complex_ else np.zeros(r, np.float32)
    E32 = 2.0 ** -24
    if complex_:
        c, ct, st, l1, l2, _ = oracle.csjac2(a11, a22, a21r, a21i)
    else:
        c, ct, l1, l2, _ = oracle.ssjac2(a11, a22, a21r)
        st = np.zeros_like(c)
    qc, qtr, qti, _, _ = oracle.q_zsjac2(a11.astype(float), a22.astype(float), a21r.astype(float),
                                         a21i.astype(float))
    cos_b = (14.000006 if complex_ else 8.000002) * E32
    tan_b = (11.500004 if complex_ else 5.500001) * E32
    et_b = (1 + 4.000001 * E32) * (1 + tan_b) * (1 + E32) - 1
    for i in range(r):
        rc = hl(qc[i])
        assert abs(D(float(c[i])) - rc) <= D(cos_b) * rc, i
        rr, ri = hl(qtr[i]), hl(qti[i])
        mag = (rr * rr + ri * ri).sqrt()
        err = ((D(float(ct[i])) - rr) ** 2 + (D(float(st[i])) - ri) ** 2).sqrt()
        assert err <= D(et_b) * mag + D(2.0 ** -149), i


def test_graded_relative_accuracy_against_twin():
    """A column-graded matrix B D: the FP64 oracle's small singular values
    relatively accurate against the twin (one-sided Jacobi's relative
    accuracy)."""
    g = np.random.default_rng(19)
    B = g.standard_normal((30, 12))
    A = np.asfortranarray(B * np.ldexp(1.0, -40 * np.arange(12)))
    o = oracle.vjsvd(A)
    t = oracle.q_vjsvd(A)
    sq = t["sigma"][:, 0]
    assert np.all(np.abs(o["sigma"] / sq - 1) <= 1e-13)

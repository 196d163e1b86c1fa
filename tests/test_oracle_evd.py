"""Pins of the oracle's batched 2x2 EVD (Listing 1 / Alg. d8jac2) against
what the paper and the mathematics fix, never against the oracle itself."""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads
from tests.exact import D, EPS, charpoly, eig2_exact, rotation_exact, ulp_step

NU = np.finfo(np.float64).max
MU = 5e-324  # the smallest subnormal


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def normal_range_inputs(r, complex_, seed=7):
    """Entries in the normal range with moderate exponents: the Eq. e:z
    power-of-two scaling is then exact, so the Prop. p:s2 bounds apply to the
    exact rotation of the input itself."""
    g = np.random.default_rng(seed)
    e = lambda: g.integers(-300, 300, size=r)
    s = lambda: np.where(g.random(r) < 0.5, -1.0, 1.0)
    a11 = np.ldexp(1 + g.random(r), e()) * s()
    a22 = np.ldexp(1 + g.random(r), e()) * s()
    a21r = np.ldexp(1 + g.random(r), e()) * s()
    a21i = np.ldexp(1 + g.random(r), e()) * s() if complex_ else np.zeros(r)
    # also near-equal diagonals (tan(2 phi) large) and tiny off-diagonals
    k = r // 4
    a22[:k] = a11[:k] * (1 + np.ldexp(g.random(k), -40))
    a21r[k:2 * k] = np.ldexp(a21r[k:2 * k], -200)
    return a11, a22, a21r, a21i


@pytest.mark.parametrize("complex_", [False, True])
def test_prop_2_1_rotation_bounds(complex_):
    """Prop. p:s2 (Eq. e:prop): relative errors of tan(phi), cos(phi) and
    e^{i alpha} against the exact diagonalising rotation."""
    r = 400
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_)
    if complex_:
        c, ct, st, l1, l2, zp = oracle.zsjac2(a11, a22, a21r, a21i)
    else:
        c, ct, l1, l2, zp = oracle.dsjac2(a11, a22, a21r)
        st = np.zeros(r)
    tan_bound = (11.500004 if complex_ else 5.500001) * EPS
    cos_bound = (14.000006 if complex_ else 8.000002) * EPS
    # |fl(e^{ia}) fl(tan)| with one more rounding of the product
    et_bound = (1 + 4.000001 * EPS) * (1 + tan_bound) * (1 + EPS) - 1
    for i in range(r):
        t, cc, ca, sa = rotation_exact(a11[i], a22[i], a21r[i], a21i[i])
        assert abs(D(c[i]) - cc) <= D(cos_bound) * cc, i
        ex_r, ex_i = ca * t, sa * t
        err = ((D(ct[i]) - ex_r) ** 2 + (D(st[i]) - ex_i) ** 2).sqrt()
        if t != 0:
            assert err <= D(et_bound) * abs(t), i
        if not complex_:
            # real: the output is sign(a21) tan(phi) itself
            assert abs(D(ct[i]) - ca * t) <= D(tan_bound) * abs(t), i


@pytest.mark.parametrize("complex_", [False, True])
def test_eigenvalues_closed_form(complex_):
    """Eigenvalues against the closed form (a11+a22)/2 +- sqrt(...): the one
    of larger magnitude relatively, the other normwise (section SM7.1)."""
    r = 400
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_, seed=11)
    if complex_:
        _, _, _, l1, l2, zp = oracle.zsjac2(a11, a22, a21r, a21i)
    else:
        _, _, l1, l2, zp = oracle.dsjac2(a11, a22, a21r)
    for i in range(r):
        lp, lm = eig2_exact(a11[i], a22[i], a21r[i], a21i[i])
        got = sorted([D(l1[i]), D(l2[i])])
        ex = sorted([lp, lm])
        anorm = max(abs(D(a11[i])), abs(D(a22[i])), (D(a21r[i]) ** 2 + D(a21i[i]) ** 2).sqrt())
        big = 0 if abs(ex[0]) > abs(ex[1]) else 1
        assert abs(got[big] - ex[big]) <= D(16 * EPS) * abs(ex[big]), i
        assert abs(got[1 - big] - ex[1 - big]) <= D(16 * EPS) * anorm, i
        # the permutation bit: p = 1 iff lambda1' < lambda2'
        assert (zp[i] & 1) == (1 if D(l1[i]) < D(l2[i]) else 0)


def test_charpoly_brute_force_real():
    """Tiny dyadic real matrices: p(lambda) = lambda^2 - tr lambda + det,
    evaluated exactly, changes sign within 4 ulp of each computed eigenvalue."""
    vals = [0.0, 0.5, -0.5, 1.0, -1.0, 2.0, -2.0, 3.0, -3.0]
    trip = list(itertools.product(vals, repeat=3))
    a11, a22, a21 = (np.array(x) for x in zip(*trip))
    _, _, l1, l2, _ = oracle.dsjac2(a11, a22, a21)
    for i in range(len(trip)):
        _check_roots(a11[i], a22[i], a21[i], 0.0, l1[i], l2[i])


def test_charpoly_brute_force_complex():
    vals = [0.0, 0.5, -1.0, 2.0, -3.0]
    quad = list(itertools.product(vals, repeat=4))
    a11, a22, a21r, a21i = (np.array(x) for x in zip(*quad))
    _, _, _, l1, l2, _ = oracle.zsjac2(a11, a22, a21r, a21i)
    for i in range(len(quad)):
        _check_roots(a11[i], a22[i], a21r[i], a21i[i], l1[i], l2[i])


def _check_roots(a11, a22, ar, ai, l1, l2):
    if ar == 0 and ai == 0 and a11 == a22:
        assert l1 == a11 and l2 == a22
        return
    # the root of larger magnitude within 4 ulp; the other one normwise
    # (within 8 eps ||A||_max), as section SM7.1 states for lambda_min
    anorm = max(abs(a11), abs(a22), math.hypot(ar, ai))
    big = l1 if abs(l1) >= abs(l2) else l2
    for lam in (l1, l2):
        if charpoly(a11, a22, ar, ai, lam) == 0:
            continue
        if lam is big:
            lo, hi = ulp_step(lam, -4), ulp_step(lam, 4)
        else:
            lo, hi = lam - 8 * EPS * anorm, lam + 8 * EPS * anorm
        plo, phi = charpoly(a11, a22, ar, ai, lo), charpoly(a11, a22, ar, ai, hi)
        assert plo * phi <= 0, (a11, a22, ar, ai, lam)
    # the two computed values are the two distinct roots
    assert abs((l1 + l2) - (a11 + a22)) <= 8 * EPS * (abs(a11) + abs(a22) + abs(ar) + abs(ai))


@pytest.mark.parametrize("complex_", [False, True])
def test_residual_and_orientation(complex_):
    """U from Eq. e:1 built from the outputs, U = cos(phi) [[1, -conj(e)],
    [e, 1]], e = e^{i alpha} tan(phi), diagonalises A: ||A U - U Lambda||
    is a few eps of ||A||.  A wrong sign, conjugation or index fails it."""
    r = 300
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_, seed=13)
    if complex_:
        c, ct, st, l1, l2, _ = oracle.zsjac2(a11, a22, a21r, a21i)
    else:
        c, ct, l1, l2, _ = oracle.dsjac2(a11, a22, a21r)
        st = np.zeros(r)
    for i in range(r):
        cc, er, ei = D(c[i]), D(ct[i]), D(st[i])
        A = [[(D(a11[i]), D(0)), (D(a21r[i]), -D(a21i[i]))],
             [(D(a21r[i]), D(a21i[i])), (D(a22[i]), D(0))]]
        U = [[(cc, D(0)), (-cc * er, cc * ei)], [(cc * er, cc * ei), (cc, D(0))]]
        lam = [D(l1[i]), D(l2[i])]
        worst = D(0)
        for row in range(2):
            for col in range(2):
                sr = si = D(0)
                for k in range(2):
                    xr, xi = A[row][k]
                    yr, yi = U[k][col]
                    sr += xr * yr - xi * yi
                    si += xr * yi + xi * yr
                ur, ui = U[row][col]
                sr -= ur * lam[col]
                si -= ui * lam[col]
                worst = max(worst, (sr * sr + si * si).sqrt())
        anorm = max(abs(D(a11[i])), abs(D(a22[i])), (D(a21r[i]) ** 2 + D(a21i[i]) ** 2).sqrt())
        assert worst <= D(32 * EPS) * anorm, i


def test_offdiagonal_zero():
    """a21 = 0: tan(phi) = +-0, cos(phi) = 1, lambda = (a11, a22) exactly."""
    g = np.random.default_rng(3)
    a11 = g.standard_normal(100) * 10.0 ** g.integers(-30, 30, 100)
    a22 = g.standard_normal(100) * 10.0 ** g.integers(-30, 30, 100)
    z = np.zeros(100)
    c, t, l1, l2, _ = oracle.dsjac2(a11, a22, z)
    assert np.all(c == 1.0) and np.all(t == 0.0)
    assert np.array_equal(l1, a11) and np.array_equal(l2, a22)
    c, ct, st, l1, l2, _ = oracle.zsjac2(a11, a22, z, z)
    assert np.all(c == 1.0) and np.all(ct == 0.0) and np.all(st == 0.0)
    assert np.array_equal(l1, a11) and np.array_equal(l2, a22)


def test_equal_diagonal():
    """a11 = a22, a21 != 0: |tan(phi)| = 1, cos(phi) = fl(1/fl(sqrt 2))."""
    g = np.random.default_rng(4)
    a = g.standard_normal(100) * 10.0 ** g.integers(-100, 100, 100)
    b = g.standard_normal(100) * 10.0 ** g.integers(-100, 100, 100)
    c, t, _, _, _ = oracle.dsjac2(a, a, b)
    assert np.all(np.abs(t) == 1.0)
    assert np.all(c == 1.0 / math.sqrt(2.0))
    assert np.all(np.sign(t) == np.sign(b))


def test_evil_matrix():
    """Eq. e:evil: [[nu/8, mu - i mu], [mu + i mu, nu/8]] gives
    fl(e^{i alpha}) = 1 + i, fl(tan phi) = 1, fl(cos phi) = fl(1/fl(sqrt 2)),
    zeta = 0."""
    for sgn in (1.0, -1.0):
        c, ct, st, l1, l2, zp = oracle.zsjac2([NU / 8], [NU / 8], [MU], [sgn * MU])
        assert ct[0] == 1.0 and st[0] == sgn
        assert c[0] == 1.0 / math.sqrt(2.0)
        assert (zp[0] >> 1) == 0


def test_zero_matrix():
    c, ct, st, l1, l2, zp = oracle.zsjac2([0.0], [0.0], [0.0], [0.0])
    assert c[0] == 1.0 and ct[0] == 0.0 and st[0] == 0.0 and l1[0] == 0.0 and l2[0] == 0.0
    assert (zp[0] >> 1) == -2094 and (zp[0] & 1) == 0


def test_scaling_exponent_cases():
    """Eq. e:z: zeta = eta - floor(lg max|component|), eta = 1020, packed as
    (zeta' << 1) | p with zeta' = -zeta."""
    cases = [(1.0, 0.0, 0.0, 0.0, 1020), (2.0, 0.0, 0.0, 0.0, 1019), (0.0, 0.0, 0.75, 0.0, 1021),
             (NU, 0.0, 0.0, 0.0, -3), (MU, 0.0, 0.0, 0.0, 2094), (0.0, 0.0, 0.0, 3.0, 1019),
             (1.0, 8.0, -0.5, 4.0, 1017)]
    for a11, a22, ar, ai, zeta in cases:
        _, _, _, _, _, zp = oracle.zsjac2([a11], [a22], [ar], [ai])
        assert (zp[0] >> 1) == -zeta, (a11, a22, ar, ai)


def test_complex_on_real_input_bit_equals_real():
    """Supplement SM2.1: the complex algorithm on a real input returns the
    real algorithm's outputs bit for bit (Im a21 = +0)."""
    a11, a22, a21 = workloads.evd_batch(1 << 14, False)
    c1, t1, l11, l21, zp1 = oracle.dsjac2(a11, a22, a21)
    c2, ct2, st2, l12, l22, zp2 = oracle.zsjac2(a11, a22, a21, np.zeros_like(a21))
    for x, y in ((c1, c2), (t1, ct2), (l11, l12), (l21, l22)):
        assert np.array_equal(x.view(np.uint64), y.view(np.uint64))
    assert np.array_equal(zp1, zp2)
    assert np.all(st2 == 0.0)


@pytest.mark.parametrize("complex_", [False, True])
def test_wide_range_outputs_finite(complex_):
    """Prop. p:s2: after the Eq. e:z scaling nothing avoidable overflows, for
    entries anywhere from subnormal to near DBL_MAX and exact zeros."""
    b = workloads.evd_batch(1 << 15, complex_)
    if complex_:
        c, ct, st, l1, l2, zp = oracle.zsjac2(*b)
        s1, s2 = oracle.zsjac2_scaled(*b)
        outs = (c, ct, st)
    else:
        c, ct, l1, l2, zp = oracle.dsjac2(*b)
        s1, s2 = oracle.zsjac2_scaled(b[0], b[1], b[2], np.zeros_like(b[2]))
        outs = (c, ct)
    for o in outs + (s1, s2):
        assert np.all(np.isfinite(o))
    assert np.all((c > 0.7) & (c <= 1.0))
    z = -(zp >> 1)
    assert np.all((z >= -3) & (z <= 2094))
    # the backscaled eigenvalues are 2^-zeta lambda' up to one rounding
    ref1 = np.ldexp(s1, -z)
    assert np.array_equal(ref1, l1)


def test_prescribed_eigenvalue_batch():
    """The paper's test data (Eq. e:2 construction): every output finite and
    the residual small for matrices built from prescribed eigenvalues."""
    a11, a22, a21r, a21i = workloads.evd_prescribed(2000, True)
    c, ct, st, l1, l2, _ = oracle.zsjac2(a11, a22, a21r, a21i)
    assert np.all(np.isfinite(c)) and np.all(np.isfinite(ct)) and np.all(np.isfinite(st))
    e = ct + 1j * st
    # |e^{i alpha}| tan(phi) <= 1 (|tan phi| <= 1), up to rounding
    assert np.all(np.abs(e) <= 1.0 + 32 * EPS)

"""Pins of the oracle's single precision 2x2 EVD (Listing 1 / Alg. d8jac2
with the binary32 constants of section 2.4: nu = FLT_MAX, fl(sqrt nu) =
1.844674297E+19, mu = FLT_TRUE_MIN, eta = FLT_MAX_EXP - 4) against exact
arithmetic and the special cases the paper fixes.  Prop. p:s2 holds for any
precision with p >= 23, with eps = 2^-24 here."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_08361_gb300 import workloads
from tests.exact import D, charpoly, eig2_exact, rotation_exact

EPS = 2.0 ** -24
FMAX = float(np.finfo(np.float32).max)
FMIN = float(np.float32(2.0 ** -149))


def f32(x):
    return np.asarray(x, dtype=np.float32)


def normal_range_inputs(r, complex_, seed=7):
    g = np.random.default_rng(seed)
    e = lambda: g.integers(-40, 40, size=r)
    s = lambda: np.where(g.random(r) < 0.5, -1.0, 1.0)
    m = lambda: 1 + np.ldexp(g.integers(0, 1 << 23, size=r).astype(float), -23)
    a11 = f32(np.ldexp(m(), e()) * s())
    a22 = f32(np.ldexp(m(), e()) * s())
    a21r = f32(np.ldexp(m(), e()) * s())
    a21i = f32(np.ldexp(m(), e()) * s()) if complex_ else np.zeros(r, np.float32)
    k = r // 4
    a22[:k] = f32(a11[:k].astype(float) * (1 + np.ldexp(g.integers(1, 64, k).astype(float), -20)))
    a21r[k:2 * k] = f32(np.ldexp(a21r[k:2 * k].astype(float), -30))
    return a11, a22, a21r, a21i


def run(a11, a22, a21r, a21i, complex_):
    if complex_:
        return oracle.csjac2(a11, a22, a21r, a21i)
    c, t, l1, l2, zp = oracle.ssjac2(a11, a22, a21r)
    return c, t, np.zeros_like(c), l1, l2, zp


@pytest.mark.parametrize("complex_", [False, True])
def test_prop_2_1_rotation_bounds(complex_):
    r = 400
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_)
    c, ct, st, l1, l2, zp = run(a11, a22, a21r, a21i, complex_)
    tan_bound = (11.500004 if complex_ else 5.500001) * EPS
    cos_bound = (14.000006 if complex_ else 8.000002) * EPS
    et_bound = (1 + 4.000001 * EPS) * (1 + tan_bound) * (1 + EPS) - 1
    for i in range(r):
        t, cc, ca, sa = rotation_exact(float(a11[i]), float(a22[i]), float(a21r[i]), float(a21i[i]))
        assert abs(D(float(c[i])) - cc) <= D(cos_bound) * cc, i
        err = ((D(float(ct[i])) - ca * t) ** 2 + (D(float(st[i])) - sa * t) ** 2).sqrt()
        if t != 0:
            assert err <= D(et_bound) * abs(t), i


@pytest.mark.parametrize("complex_", [False, True])
def test_eigenvalues_closed_form(complex_):
    r = 400
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_, seed=11)
    c, ct, st, l1, l2, zp = run(a11, a22, a21r, a21i, complex_)
    for i in range(r):
        lp, lm = eig2_exact(float(a11[i]), float(a22[i]), float(a21r[i]), float(a21i[i]))
        got = sorted([D(float(l1[i])), D(float(l2[i]))])
        ex = sorted([lp, lm])
        anorm = max(abs(D(float(a11[i]))), abs(D(float(a22[i]))),
                    (D(float(a21r[i])) ** 2 + D(float(a21i[i])) ** 2).sqrt())
        big = 0 if abs(ex[0]) > abs(ex[1]) else 1
        assert abs(got[big] - ex[big]) <= D(16 * EPS) * abs(ex[big]), i
        assert abs(got[1 - big] - ex[1 - big]) <= D(16 * EPS) * anorm, i
        assert (zp[i] & 1) == (1 if l1[i] < l2[i] else 0)


def f32_step(x, k):
    x = np.float32(x)
    for _ in range(abs(k)):
        x = np.nextafter(x, np.float32(np.inf if k > 0 else -np.inf))
    return float(x)


@pytest.mark.parametrize("complex_", [False, True])
def test_charpoly_brute_force(complex_):
    """Tiny dyadic matrices: p(lambda), exact in rationals, changes sign
    within 4 binary32 ulps of the larger computed eigenvalue and within
    8 eps ||A|| of the other."""
    vals = [0.0, 0.5, -1.0, 2.0, -3.0] if complex_ else [0.0, 0.5, -0.5, 1.0, -1.0, 2.0, -3.0]
    combos = list(itertools.product(vals, repeat=4 if complex_ else 3))
    cols = [f32(x) for x in zip(*combos)]
    if not complex_:
        cols.append(np.zeros(len(combos), np.float32))
    _, _, _, l1, l2, _ = run(*cols, complex_)
    for i in range(len(combos)):
        a11, a22, ar, ai = (float(c[i]) for c in cols)
        L1, L2 = float(l1[i]), float(l2[i])
        if ar == 0 and ai == 0 and a11 == a22:
            assert L1 == a11 and L2 == a22
            continue
        anorm = max(abs(a11), abs(a22), math.hypot(ar, ai))
        big = L1 if abs(L1) >= abs(L2) else L2
        for lam in (L1, L2):
            if charpoly(a11, a22, ar, ai, lam) == 0:
                continue
            if lam is big:
                lo, hi = f32_step(lam, -4), f32_step(lam, 4)
            else:
                lo, hi = lam - 8 * EPS * anorm, lam + 8 * EPS * anorm
            assert charpoly(a11, a22, ar, ai, lo) * charpoly(a11, a22, ar, ai, hi) <= 0, combos[i]


@pytest.mark.parametrize("complex_", [False, True])
def test_residual_and_orientation(complex_):
    r = 300
    a11, a22, a21r, a21i = normal_range_inputs(r, complex_, seed=13)
    c, ct, st, l1, l2, _ = run(a11, a22, a21r, a21i, complex_)
    for i in range(r):
        cc, er, ei = D(float(c[i])), D(float(ct[i])), D(float(st[i]))
        A = [[(D(float(a11[i])), D(0)), (D(float(a21r[i])), -D(float(a21i[i])))],
             [(D(float(a21r[i])), D(float(a21i[i]))), (D(float(a22[i])), D(0))]]
        U = [[(cc, D(0)), (-cc * er, cc * ei)], [(cc * er, cc * ei), (cc, D(0))]]
        lam = [D(float(l1[i])), D(float(l2[i]))]
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
        anorm = max(abs(D(float(a11[i]))), abs(D(float(a22[i]))),
                    (D(float(a21r[i])) ** 2 + D(float(a21i[i])) ** 2).sqrt())
        assert worst <= D(32 * EPS) * anorm, i


def test_special_cases():
    """a21 = 0: tan = 0, cos = 1, lambda = (a11, a22) exactly; a11 = a22:
    |tan| = 1, cos = fl(1/fl(sqrt 2)) in binary32."""
    g = np.random.default_rng(3)
    a11 = f32(g.standard_normal(100) * 10.0 ** g.integers(-10, 10, 100))
    a22 = f32(g.standard_normal(100) * 10.0 ** g.integers(-10, 10, 100))
    z = np.zeros(100, np.float32)
    c, t, l1, l2, _ = oracle.ssjac2(a11, a22, z)
    assert np.all(c == 1.0) and np.all(t == 0.0)
    assert np.array_equal(l1, a11) and np.array_equal(l2, a22)
    c, t, _, _, _ = oracle.ssjac2(a11, a11, a22)
    r2 = np.float32(1.0) / np.sqrt(np.float32(2.0))
    assert np.all(np.abs(t) == 1.0) and np.all(c == r2)


def test_evil_matrix():
    """Eq. e:evil in binary32: [[nu/8, mu - i mu], [mu + i mu, nu/8]] gives
    e^{i alpha} tan(phi) = 1 + i, cos(phi) = fl(1/fl(sqrt 2)), zeta = 0."""
    for sgn in (1.0, -1.0):
        c, ct, st, l1, l2, zp = oracle.csjac2([FMAX / 8], [FMAX / 8], [FMIN], [sgn * FMIN])
        assert ct[0] == 1.0 and st[0] == sgn
        assert c[0] == np.float32(1.0) / np.sqrt(np.float32(2.0))
        assert (zp[0] >> 1) == 0


def test_scaling_exponent_cases():
    """Eq. e:z with eta = FLT_MAX_EXP - 4 = 124; zero gives 273 (the frexp
    exponent of FLT_TRUE_MIN)."""
    cases = [(1.0, 0.0, 0.0, 0.0, 124), (2.0, 0.0, 0.0, 0.0, 123), (0.0, 0.0, 0.75, 0.0, 125),
             (FMAX, 0.0, 0.0, 0.0, -3), (FMIN, 0.0, 0.0, 0.0, 273), (0.0, 0.0, 0.0, 0.0, 273),
             (1.0, 8.0, -0.5, 4.0, 121)]
    for a11, a22, ar, ai, zeta in cases:
        *_, zp = oracle.csjac2([a11], [a22], [ar], [ai])
        assert (zp[0] >> 1) == -zeta, (a11, a22, ar, ai)


def test_complex_on_real_input_bit_equals_real():
    a11, a22, a21 = workloads.evd_batch_f32(1 << 14, False)
    c1, t1, l11, l21, zp1 = oracle.ssjac2(a11, a22, a21)
    c2, ct2, st2, l12, l22, zp2 = oracle.csjac2(a11, a22, a21, np.zeros_like(a21))
    for x, y in ((c1, c2), (t1, ct2), (l11, l12), (l21, l22)):
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    assert np.array_equal(zp1, zp2) and np.all(st2 == 0.0)


@pytest.mark.parametrize("complex_", [False, True])
def test_wide_range_outputs_finite(complex_):
    """Prop. p:s2 in binary32: entries from subnormal to near FLT_MAX and
    exact zeros never give a non-finite rotation."""
    b = workloads.evd_batch_f32(1 << 15, complex_)
    if complex_:
        c, ct, st, l1, l2, zp = oracle.csjac2(*b)
        outs = (c, ct, st)
    else:
        c, ct, l1, l2, zp = oracle.ssjac2(*b)
        outs = (c, ct)
    for o in outs:
        assert np.all(np.isfinite(o))
    assert np.all((c > 0.7) & (c <= 1.0))
    z = -(zp >> 1)
    assert np.all((z >= -3) & (z <= 273))

"""Pins of the oracle's wide-exponent Frobenius norm (Alg. rnF, supplement
SM6, one lane): against the exact norm (rationals and 80-digit decimals)
where the double result would overflow or underflow, and against the
identities the (e, f) arithmetic must keep."""
from decimal import Decimal
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.exact import D

U = 2.0 ** -53
NU = np.finfo(np.float64).max
MU = 5e-324


def exact_norm(x):
    s = sum(Fraction(float(v)) ** 2 for v in x)
    return D(s).sqrt()


def ef_value(e, f):
    if e == -np.inf:
        return Decimal(0)
    return D(f) * (Decimal(2) ** int(e))


def check(x, slack=2):
    e, f = oracle.rnF(x)
    assert 1.0 <= f < 2.0 or (e == -np.inf and f == 1.0)
    assert e == -np.inf or e == int(e)
    ex = exact_norm(x)
    got = ef_value(e, f)
    if ex == 0:
        assert got == 0
        return
    assert abs(got - ex) <= Decimal((len(x) + slack) * U) * ex, (got, ex)


@pytest.mark.parametrize("seed", range(4))
def test_random_moderate(seed):
    g = np.random.default_rng(seed)
    check(g.standard_normal(300) * np.exp2(g.integers(-30, 30, 300)))


def test_beyond_the_double_range():
    """||nu 1|| = nu sqrt(m) overflows as a double but not as (e, f); a
    vector of subnormals underflows when squared but not here."""
    check(np.full(5, NU))
    check(np.full(7, MU))
    check(np.array([NU, NU / 3, 1.0, MU, -NU]))
    check(np.array([MU, 3 * MU, -7 * MU, 2.0 ** -1060]))
    e, f = oracle.rnF(np.full(4, NU))
    assert e == 1024 and f == float(np.nextafter(2.0, 0))  # 2 nu exactly
    assert oracle.rnF(np.full(4, MU)) == (-1073.0, 1.0)  # 2 mu exactly


def test_zero_and_single_entry():
    """0 = (-inf, 1); one entry x gives (floor(lg|x|), |x| / 2^floor(lg|x|))
    exactly, since sqrt(RN(f^2)) = f in binary floating point."""
    assert oracle.rnF(np.zeros(9)) == (-np.inf, 1.0)
    g = np.random.default_rng(5)
    for x in list(g.standard_normal(50) * np.exp2(g.integers(-1070, 1020, 50))) + [NU, -MU, 1.0]:
        e, f = oracle.rnF([0.0, x, 0.0])
        m, k = np.frexp(abs(x))
        assert (e, f) == (float(k - 1), 2 * m), x


def test_scale_invariance():
    """rnF(2^k x) = (e + k, f) exactly: the (e, f) steps act on exponent
    differences only (entries with 20 significant bits stay exact when
    scaled into the subnormal range)."""
    g = np.random.default_rng(7)
    x = np.ldexp(g.integers(-(1 << 20), 1 << 20, 64).astype(float), -20)
    e0, f0 = oracle.rnF(x)
    for k in (-1030, -600, -1, 1, 300, 1000):
        e, f = oracle.rnF(np.ldexp(x, k))
        assert (e, f) == (e0 + k, f0), k


def test_order_of_magnitude_mix():
    """Entries spanning the whole double range: the tiny ones are negligible
    and the result is the norm of the large ones."""
    x = np.array([1e300, 1e-300, 3e299, MU, 0.0, -2e300])
    check(x)

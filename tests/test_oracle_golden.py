"""The oracle against the values the paper prints for its worked examples
(tests/golden/paper_examples.txt, each line citing where the paper gives
it)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
NU = np.finfo(np.float64).max
MU = np.float64(5e-324)


def load():
    table = {}
    with open(os.path.join(HERE, "golden", "paper_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, cite, vals = (x.strip() for x in line.split("|"))
            assert cite, name
            table[name] = vals.split()
    return table


G = load()


def num(tok):
    if tok.startswith("sqrt(") and tok.endswith(")"):
        return math.sqrt(float(tok[5:-1]))
    if tok.startswith("1/sqrt(") and tok.endswith(")"):
        return 1.0 / math.sqrt(float(tok[7:-1]))
    return float(Fraction(tok))


def test_fixture_file_complete():
    for k in ("spectrum_xi_m3_n4", "ef_of_12", "ef_sqrt_80", "evil_cos", "eta_f32", "sqrt_nu_f32"):
        assert k in G


def test_spectrum_example():
    """A diagonal matrix built from Sigma[-3, 4, I_4] with its columns in a
    scrambled order: the oracle's SVD returns the printed diagonal, sorted
    non-increasingly, exactly."""
    s = [num(t) for t in G["spectrum_xi_m3_n4"]]
    perm = [2, 0, 3, 1]
    A = np.zeros((5, 4))
    for j, p in enumerate(perm):
        A[j, j] = s[p]
    r = oracle.vjsvd(A)
    assert r["sigma"].tolist() == sorted(s, reverse=True)


@pytest.mark.parametrize("which,x", [("12", [2.0, 2.0, 2.0]), ("80", [4.0, 8.0])])
def test_ef_examples(which, x):
    """Alg. rnF on vectors whose squared norms are 12 and 80: the square
    root of the printed (e, f) is the printed (e'', f'')."""
    e2, f2 = (num(t) for t in G["ef_of_" + which])
    assert sum(v * v for v in x) == 2.0 ** e2 * f2
    e, f = oracle.rnF(np.array(x))
    want_e, want_f = (num(t) for t in G["ef_sqrt_" + which])
    assert e == want_e and f == want_f


def test_evil_matrix():
    for sgn in (1.0, -1.0):
        c, ct, st, l1, l2, zp = oracle.zsjac2([NU / 8], [NU / 8], [MU], [sgn * MU])
        assert -(int(zp[0]) >> 1) == num(G["evil_zeta"][0])
        assert math.hypot(ct[0], st[0]) == math.hypot(*[num(t) for t in G["evil_exp_ialpha"]])
        assert ct[0] == num(G["evil_tan"][0]) * num(G["evil_exp_ialpha"][0])
        assert st[0] == sgn * num(G["evil_exp_ialpha"][1])
        assert c[0] == num(G["evil_cos"][0])


def test_eta_f64():
    """zeta = eta - floor(lg max |a_ij|): a matrix with largest entry 1 has
    zeta = eta."""
    _, _, _, _, zp = oracle.dsjac2([1.0], [0.5], [0.25])
    assert -(int(zp[0]) >> 1) == int(G["eta_f64"][0])


def test_eta_f32():
    _, _, _, _, zp = oracle.ssjac2([1.0], [0.5], [0.25])
    assert -(int(zp[0]) >> 1) == int(G["eta_f32"][0])


def test_sqrt_nu_constants():
    """The printed fl(sqrt(nu)) are the correctly rounded square roots of
    DBL_MAX and FLT_MAX (checked exactly with integers), and the printed
    eta are the exponent bounds stated beside them."""
    v = float(G["sqrt_nu_f64"][0])
    q = Fraction(v)
    nu = Fraction(NU)
    # v is the double nearest to sqrt(nu): v^2 <= nu < next(v)^2 or closest
    lo, hi = Fraction(np.nextafter(v, 0)), Fraction(np.nextafter(v, np.inf))
    assert abs(q * q - nu) <= abs(lo * lo - nu) and abs(q * q - nu) <= abs(hi * hi - nu)
    v32 = np.float32(G["sqrt_nu_f32"][0])
    nu32 = Fraction(float(np.finfo(np.float32).max))
    q32 = Fraction(float(v32))
    lo32 = Fraction(float(np.nextafter(v32, np.float32(0))))
    hi32 = Fraction(float(np.nextafter(v32, np.float32(np.inf))))
    assert abs(q32 * q32 - nu32) <= abs(lo32 * lo32 - nu32)
    assert abs(q32 * q32 - nu32) <= abs(hi32 * hi32 - nu32)
    # floor(lg(nu/8)) from the exact binary exponent (a float log2 of a
    # value just below 2^1021 rounds up to 1021)
    assert int(G["eta_f64"][0]) == math.frexp(NU / 8)[1] - 1
    assert int(G["eta_f32"][0]) == math.frexp(float(np.finfo(np.float32).max) / 8)[1] - 1

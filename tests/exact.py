"""Exact and high-precision references for the oracle pins (stdlib only).

Everything here is computed from the mathematical definition (rationals
via fractions.Fraction, square roots via decimal at 80 digits), never from
the oracle or the CUDA library.
"""
from decimal import Decimal, getcontext
from fractions import Fraction
import math

getcontext().prec = 80

EPS = 2.0 ** -53  # the paper's epsilon, half an ulp of 1


def D(x) -> Decimal:
    """Exact Decimal of a double or Fraction."""
    if isinstance(x, Fraction):
        return Decimal(x.numerator) / Decimal(x.denominator)
    return Decimal(Fraction(float(x)).numerator) / Decimal(Fraction(float(x)).denominator)


def eig2_exact(a11, a22, a21r, a21i=0.0):
    """Exact eigenvalues (lam_plus, lam_minus) of the Hermitian 2x2 matrix,
    closed form (a11+a22)/2 +- sqrt(((a11-a22)/2)^2 + |a21|^2), in Decimal."""
    h = (D(a11) + D(a22)) / 2
    d = (D(a11) - D(a22)) / 2
    r = (d * d + D(a21r) ** 2 + D(a21i) ** 2).sqrt()
    return h + r, h - r


def rotation_exact(a11, a22, a21r, a21i=0.0):
    """Exact (tan(phi), cos(phi), cos(alpha), sin(alpha)) of the diagonalising
    rotation of Eq. e:1: tan(2 phi) = 2|a21|/(a11 - a22), phi in [-pi/4, pi/4],
    alpha = arg a21 (arg 0 = 0)."""
    aa = (D(a21r) ** 2 + D(a21i) ** 2).sqrt()
    a = D(a11) - D(a22)
    if aa == 0:
        t = Decimal(0)
    elif a == 0:
        t = Decimal(1)
    else:
        t2 = 2 * aa / a
        t = t2 / (1 + (1 + t2 * t2).sqrt())
    c = 1 / (1 + t * t).sqrt()
    if aa == 0:
        ca, sa = Decimal(1), Decimal(0)
    else:
        ca, sa = D(a21r) / aa, D(a21i) / aa
    return t, c, ca, sa


def charpoly(a11, a22, a21r, a21i, lam) -> Fraction:
    """p(lam) = lam^2 - tr(A) lam + det(A), exactly in rationals."""
    A11, A22 = Fraction(a11), Fraction(a22)
    B = Fraction(a21r) ** 2 + Fraction(a21i) ** 2
    L = Fraction(lam)
    return L * L - (A11 + A22) * L + (A11 * A22 - B)


def ulp_step(x: float, k: int) -> float:
    """x moved by k ulps (k may be negative)."""
    for _ in range(abs(k)):
        x = math.nextafter(x, math.inf if k > 0 else -math.inf)
    return x


def ordered(x: float) -> int:
    """Map a double to an integer in the same order (ulp metric); +-0 -> 0."""
    import struct
    i = struct.unpack("<q", struct.pack("<d", float(x)))[0]
    return i if i >= 0 else -(i & 0x7FFFFFFFFFFFFFFF)

// fp64sel.cuh -- forms of fp64soft.cuh's binary64 division, square root and
// x 2^k for the SVD step's warp-parallel rotation: written with selects
// instead of data-dependent branches (its lanes run different operations),
// and, for operands that every lane shares, x 2^k as an exponent add and an
// exact scaled comparison.  Host and device, like fp64soft.cuh; the results
// are checked on the host against IEEE arithmetic and on the GPU against the
// FP64 pipe.
#pragma once
#include "fp64soft.cuh"

namespace jsvd {
namespace soft {

// Where the lanes of a warp run different operations (the rotation puts
// independent divisions and square roots of one pair on different lanes),
// lanes that take different sides of a branch run them one after the
// other; the select-based forms have one path, so the latency of a
// dependent chain is that of one routine.  Their results are those of
// div_rn, sqrt_rn and ldexp_rn, bit for bit.

// |x| (nonzero bits u without sign, or 0) as m 2^(e - 52), m in [2^52, 2^53)
// (u = 0 gives m = 0)
SOFT_FN void unpack_sel(uint64_t u, uint64_t &m, int &e)
{
  const int E = (int)(u >> 52);
  const int lz = clz64(u) - 11;
  m = E ? ((u & kMan) | kOne52) : (u << (lz & 63));
  e = E ? E - 1023 : -1022 - lz;
}

SOFT_FN double round_pack_sel(uint64_t sign, uint64_t Q, bool sticky, int e)
{
  int sh = 3 + ((e < -1022) ? (-1022 - e) : 0);
  sh = (sh > 60) ? 60 : sh;
  const uint64_t keep = Q >> sh;
  const uint64_t half = 1ull << (sh - 1);
  const uint64_t rem = Q & ((1ull << sh) - 1ull);
  const bool up = (rem > half) || (rem == half && (sticky || (keep & 1ull)));
  const uint64_t mant = keep + (up ? 1ull : 0ull);
  const int E = e + 1023;
  const uint64_t b = (((uint64_t)(E - 1)) << 52) + mant;
  const uint64_t inf = 0x7FF0000000000000ull;
  const uint64_t r = (e < -1022) ? mant : (E >= 2047 || (b >> 52) >= 2047) ? inf : b;
  return as_f64(sign | r);
}

// Correctly rounded a / b; a, b finite, b != 0 (a zero b gives some value).
SOFT_FN double div_rn_sel(double a, double b)
{
  const uint64_t ub = as_u64(b), ua = as_u64(a);
  uint64_t d, n;
  int eb, ea;
  unpack_sel(ub & ~kSgn, d, eb);
  const uint64_t y = recip115(d);
  const uint64_t sign = (ua & kSgn) ^ (ub & kSgn);
  const uint64_t xa = ua & ~kSgn;
  unpack_sel(xa, n, ea);
  const bool lt = n < d;  // n/d in [1, 2)
  n = lt ? (n << 1) : n;
  const int e = ea - eb - (lt ? 1 : 0);
  const uint64_t hi = mulhi(n, y), lo = n * y;
  uint64_t Q = (hi << 4) | (lo >> 60);
  int64_t R = (int64_t)((n << 55) - Q * d);
  const bool neg = R < 0;
  Q = neg ? Q - 1 : Q;
  R = neg ? R + (int64_t)d : R;
  const bool big = R >= (int64_t)d;
  Q = big ? Q + 1 : Q;
  R = big ? R - (int64_t)d : R;
  const double r = round_pack_sel(sign, Q, R != 0, e);
  return (xa == 0ull) ? as_f64(sign) : r;
}

// Correctly rounded sqrt(x), x finite >= 0 (-0 gives -0).
SOFT_FN double sqrt_rn_sel(double x)
{
  const uint64_t ux = as_u64(x);
  uint64_t m;
  int e;
  unpack_sel(ux & ~kSgn, m, e);
  const bool odd = (e & 1) != 0;
  const uint64_t mt = odd ? (m << 1) : m;
  const int eh = (odd ? e - 1 : e) / 2;
  uint64_t z = rsqrt_seed(m, odd);
  {  // the third-order step of sqrt_rn
    const uint64_t wh = mulhi(z, z);
    const uint64_t p = mulhi(mt << 10, wh);
    const int64_t e60 = (int64_t)((1ull << 60) - p);
    const uint64_t a = (uint64_t)(e60 < 0 ? -e60 : e60) << 24;
    const int64_t q = (int64_t)(3ull * (mulhi(a, a) >> 46));
    const int64_t t = mulhi_s(z, (e60 + q) * 8);
    z = z + (uint64_t)t;
  }
  uint64_t S = mulhi(mt << 4, z);
  int64_t R = (int64_t)((mt << 58) - S * S);
  const bool neg = R < 0;
  R = neg ? R + (int64_t)(2 * S - 1) : R;
  S = neg ? S - 1 : S;
  const bool big = R > (int64_t)(2 * S);
  R = big ? R - (int64_t)(2 * S + 1) : R;
  S = big ? S + 1 : S;
  const double r = round_pack_sel(ux & kSgn, S, R != 0, eh);
  return ((ux & ~kSgn) == 0ull) ? x : r;
}

// x 2^k rounded to nearest-even (exact unless the result is subnormal); x
// finite, |k| < 4096.  The values of ldexp_rn (fp64bits.cuh).
SOFT_FN double ldexp_rn_sel(double x, int k)
{
  const uint64_t u = as_u64(x);
  const uint64_t sign = u & kSgn;
  const uint64_t a = u & ~kSgn;
  const int E = (int)(a >> 52);
  const int lz = clz64(a) - 11;
  const uint64_t sig = E ? ((a & kMan) | kOne52) : (a << (lz & 63));
  const int E2 = (E ? E : 1 - lz) + k;
  const uint64_t normal = (((uint64_t)(E2 - 1)) << 52) + sig;
  int sh = 1 - E2;
  sh = (sh < 1) ? 1 : (sh > 63) ? 63 : sh;
  uint64_t q = sig >> sh;
  const uint64_t rem = sig & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1);
  q += (uint64_t)((rem > half) | ((rem == half) & (q & 1ull)));
  const uint64_t r = (a == 0ull) ? 0ull
                     : (E2 >= 2047) ? 0x7FF0000000000000ull
                     : (E2 >= 1) ? normal
                     : (1 - E2 >= 54) ? 0ull
                                       : q;
  return as_f64(sign | r);
}


// ldexp_rn_sel behind a call, for the rare operands of the fast path
// below: the call keeps the compiler from evaluating it on every path.
#if defined(__CUDACC__)
static __device__ __host__ __noinline__ double ldexp_rn_call(double x, int k)
#else
static double ldexp_rn_call(double x, int k)
#endif
{
  return ldexp_rn_sel(x, k);
}

// x 2^k, the values of ldexp_rn_sel, for an x and k that every lane of the
// warp shares: when x and x 2^k are both normal the result is one integer
// add to the exponent field; otherwise (zero, subnormal, overflow) the
// select-based routine.  The branch is then taken alike by all lanes.
SOFT_FN double ldexp_rn_uni(double x, int k)
{
  const uint64_t u = as_u64(x);
  const int E = (int)((u >> 52) & 0x7FF);
  const int E2 = E + k;
  if ((unsigned)(E - 1) < 2046u && (unsigned)(E2 - 1) < 2046u)
    return as_f64(u + ((uint64_t)(int64_t)k << 52));
  return ldexp_rn_call(x, k);
}

// fl(q 2^d) > u as binary64 bit patterns (the comparison of the rounded
// product with u) for q and u positive and normal, without rounding or a
// branch: q 2^d below the normal range rounds to at most 2^-1022 <= u,
// above it overflows to infinity, and in it the exponent add is exact.
SOFT_FN bool gt_scaled_pos(double q, int d, double u)
{
  const uint64_t b = as_u64(q);
  const int E2 = (int)(b >> 52) + d;
  return (E2 >= 2047) || (E2 >= 1 && b + ((uint64_t)(int64_t)d << 52) > as_u64(u));
}

}  // namespace soft
}  // namespace jsvd

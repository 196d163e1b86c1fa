// fp64soft.cuh -- correctly rounded binary64 division and square root on
// the integer pipe (plus one FP32 reciprocal seed).
//
// GB300's FP64 pipe is narrow (~1.6 DFMA per SM per clock) and an IEEE
// division or square root costs ~8.6 DFMA there.  These routines give the
// same results bit for bit (round to nearest, ties to even, subnormal
// inputs and outputs) from 64-bit integer arithmetic:
//
//   division a/b: mantissas n/d with n/d in [1, 2); a fixed-point
//     reciprocal y ~ 2^115/d from an FP32 seed refined by one third-order
//     step y <- y (1 + eps + eps^2), eps = (2^115 - d y)/2^115; the quotient Q = floor(n 2^55 / d)
//     from Q ~ n y / 2^60 corrected with the exact remainder
//     R = n 2^55 - Q d (which fits in 64 bits), then rounded from Q's low
//     bits and R != 0 (Newton-Raphson division with an exact remainder
//     correction, as in Markstein, "IA-64 and elementary functions", 2000,
//     done here in fixed point);
//   square root of x: t = mantissa in [1, 4) with an even exponent; a
//     fixed-point inverse square root z ~ 2^63/sqrt(t) from an FP32 seed and
//     one third-order step z <- z (1 + delta/2 + 3 delta^2/8), delta =
//     1 - t z^2; S = floor(sqrt(t) 2^55)
//     from S ~ t z corrected with the exact remainder t 2^110 - S^2, then
//     rounded likewise.
//
// The routines compile for the host too (tests check them against the
// host's IEEE arithmetic).  Inputs must be finite; b != 0; x >= 0.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SOFT_FN __host__ __device__ __forceinline__
#else
#define SOFT_FN static inline
#endif

namespace jsvd {
namespace soft {

constexpr uint64_t kSgn = 0x8000000000000000ull;
constexpr uint64_t kMan = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kOne52 = 0x0010000000000000ull;

SOFT_FN uint64_t as_u64(double x)
{
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}

SOFT_FN double as_f64(uint64_t u)
{
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}

SOFT_FN uint64_t mulhi(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// high 64 bits of a (unsigned) times e (signed), |e| < 2^63
SOFT_FN int64_t mulhi_s(uint64_t a, int64_t e)
{
  const uint64_t m = mulhi(a, (uint64_t)(e < 0 ? -e : e));
  return e < 0 ? -(int64_t)m : (int64_t)m;
}

SOFT_FN int clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// |x| (finite, nonzero bits u without sign) as m 2^(e - 52), m in [2^52, 2^53)
SOFT_FN void unpack(uint64_t u, uint64_t &m, int &e)
{
  const int E = (int)(u >> 52);
  if (E) {
    m = (u & kMan) | kOne52;
    e = E - 1023;
  } else {
    const int lz = clz64(u) - 11;
    m = u << lz;
    e = -1022 - lz;
  }
}

// Round the value (Q + frac) 2^(e - 55), Q in [2^55, 2^56), frac = sticky
// (0 or nonzero below Q's last bit), to binary64 with sign; handles the
// subnormal range and overflow (to infinity).
SOFT_FN double round_pack(uint64_t sign, uint64_t Q, bool sticky, int e)
{
  // normal: 53-bit mantissa Q >> 3 at exponent e
  int sh = 3;
  if (e < -1022) sh += -1022 - e;  // subnormal: fewer mantissa bits
  if (sh > 60) sh = 60;  // below half the smallest subnormal: rounds to zero either way
  const uint64_t keep = Q >> sh;
  const uint64_t half = 1ull << (sh - 1);
  const uint64_t rem = Q & ((1ull << sh) - 1ull);
  const bool up = (rem > half) || (rem == half && (sticky || (keep & 1ull)));
  const uint64_t mant = keep + (up ? 1ull : 0ull);
  if (e < -1022) return as_f64(sign | mant);  // subnormal encoding (carry gives the min normal)
  const int E = e + 1023;
  if (E >= 2047) return as_f64(sign | 0x7FF0000000000000ull);
  // mant in [2^52, 2^53]; 2^53 carries into the exponent
  const uint64_t b = (((uint64_t)(E - 1)) << 52) + mant;
  if ((b >> 52) >= 2047) return as_f64(sign | 0x7FF0000000000000ull);
  return as_f64(sign | b);
}

// FP32 reciprocal of t = d / 2^52 in [1, 2) (t truncated to 24 bits), as a
// 64-bit fixed-point y0 ~ 2^115/d (relative error below 2^-21).
SOFT_FN uint64_t recip_seed(uint64_t d)
{
  const uint32_t tb = 0x3F800000u | (uint32_t)((d >> 29) & 0x7FFFFFu);
  float r;
#if defined(__CUDA_ARCH__)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint_as_float(tb)));
  const uint32_t rb = __float_as_uint(r);
#else
  float t;
  memcpy(&t, &tb, 4);
  r = 1.0f / t;
  uint32_t rb;
  memcpy(&rb, &r, 4);
#endif
  // r in (0.5, 1]: r = (2^23 + f) 2^(E - 150)
  const uint64_t m = 0x800000ull | (rb & 0x7FFFFFu);
  const int E = (int)((rb >> 23) & 0xFF);
  return m << (E - 150 + 63 + 0);  // r 2^63 = m 2^(E - 150 + 63)
}

// y ~ 2^115/d refined to a few units by one third-order step
// y <- y (1 + eps + eps^2), eps = (2^115 - d y) / 2^115: the seed's
// |eps| < 2^-22 leaves eps^3 < 2^-66, below the fixed-point truncations
// (a few units of y's last bit), as two Newton steps would, with one long
// multiplication fewer.
SOFT_FN uint64_t recip115(uint64_t d)
{
  const uint64_t y = recip_seed(d);
  // e = 2^115 - d y  (|e| < 2^94), as e52 = e / 2^52 = eps 2^63 in a signed word
  const uint64_t lo = d * y, hi = mulhi(d, y);  // d y < 2^116
  const uint64_t elo = 0ull - lo;
  const int64_t ehi = (int64_t)((1ull << 51) - hi - (lo != 0ull ? 1ull : 0ull));
  const int64_t e52 = (int64_t)(((uint64_t)ehi << 12) | (elo >> 52));
  // eps^2 2^63 = e52^2 / 2^63: with a = |e52| 2^21 (< 2^64), a^2 / 2^64 = e52^2 / 2^22
  const uint64_t a = (uint64_t)(e52 < 0 ? -e52 : e52) << 21;
  const int64_t e2 = (int64_t)(mulhi(a, a) >> 41);
  // y += y (eps + eps^2) = y (e52 + e2) / 2^63
  const int64_t t = mulhi_s(y, e52 + e2);  // y (e52 + e2) / 2^64
  return y + (uint64_t)(t * 2);
}

// A divisor prepared once for several quotients: its mantissa d, exponent
// and the fixed-point reciprocal y ~ 2^115/d.
struct Den {
  uint64_t sign, d, y;
  int e;
};

SOFT_FN Den prepare_den(double b)
{
  Den D;
  const uint64_t ub = as_u64(b);
  D.sign = ub & kSgn;
  unpack(ub & ~kSgn, D.d, D.e);
  D.y = recip115(D.d);
  return D;
}

// Correctly rounded a / b for a prepared divisor b (finite, != 0), a finite.
SOFT_FN double div_rn(double a, const Den &D)
{
  const uint64_t ua = as_u64(a);
  const uint64_t sign = (ua & kSgn) ^ D.sign;
  const uint64_t xa = ua & ~kSgn;
  if (xa == 0ull) return as_f64(sign);
  uint64_t n;
  int ea;
  unpack(xa, n, ea);
  const uint64_t d = D.d, y = D.y;
  int e = ea - D.e;
  if (n < d) {
    n <<= 1;  // n/d in [1, 2)
    e -= 1;
  }
  // Q ~ n 2^55 / d = n y / 2^60
  const uint64_t hi = mulhi(n, y), lo = n * y;
  uint64_t Q = (hi << 4) | (lo >> 60);
  // exact remainder R = n 2^55 - Q d (|R| < 2^63), then one fix either way:
  // y is within a few units of 2^115/d (relative 2^-60), so n y / 2^60 is
  // within 0.05 of n 2^55 / d < 2^56 and Q is off by at most one
  int64_t R = (int64_t)((n << 55) - Q * d);
  if (R < 0) {
    Q -= 1;
    R += (int64_t)d;
  }
  if (R >= (int64_t)d) {
    Q += 1;
    R -= (int64_t)d;
  }
  return round_pack(sign, Q, R != 0, e);
}

// Correctly rounded a / b.  a, b finite, b != 0.
SOFT_FN double div_rn(double a, double b) { return div_rn(a, prepare_den(b)); }

// FP32 inverse square root of t in [1, 4) (truncated to 24 bits), as a
// fixed-point z0 ~ 2^63/sqrt(t) (relative error below 2^-21).
SOFT_FN uint64_t rsqrt_seed(uint64_t m, bool twice)
{
  // t = m 2^-52 (m in [2^52, 2^53)) or 2 m 2^-52
  const uint32_t tb = ((twice ? 0x40000000u : 0x3F800000u)) | (uint32_t)((m >> 29) & 0x7FFFFFu);
  float r;
#if defined(__CUDA_ARCH__)
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__uint_as_float(tb)));
  const uint32_t rb = __float_as_uint(r);
#else
  float t;
  memcpy(&t, &tb, 4);
  r = (float)(1.0 / __builtin_sqrt((double)t));
  uint32_t rb;
  memcpy(&rb, &r, 4);
#endif
  // r in (0.5, 1]
  const uint64_t mm = 0x800000ull | (rb & 0x7FFFFFu);
  const int E = (int)((rb >> 23) & 0xFF);
  return mm << (E - 150 + 63);
}

// Correctly rounded sqrt(x), x finite >= 0 (-0 gives -0).
SOFT_FN double sqrt_rn(double x)
{
  const uint64_t ux = as_u64(x);
  if ((ux & ~kSgn) == 0ull) return x;
  uint64_t m;
  int e;
  unpack(ux, m, e);
  // x = m 2^(e - 52); make the exponent even: t = m' 2^-52 in [1, 4)
  const bool odd = (e & 1) != 0;
  const uint64_t mt = odd ? (m << 1) : m;  // < 2^54
  const int eh = (odd ? e - 1 : e) / 2;    // exact: e - odd is even
  uint64_t z = rsqrt_seed(m, odd);
  {
    // one third-order step z <- z (1 + delta/2 + 3 delta^2/8), delta =
    // 1 - t z^2 / 2^126 (|delta| < 2^-21 from the seed; the step leaves
    // about delta^3 / 3 < 2^-64, below the truncations).
    // t z^2 / 2^126 ~ 1: wh = z^2 / 2^64, p = t wh / 4 = mt wh / 2^54
    const uint64_t wh = mulhi(z, z);
    const uint64_t p = mulhi(mt << 10, wh);           // mt 2^10 wh / 2^64 = mt wh / 2^54
    const int64_t e60 = (int64_t)((1ull << 60) - p);  // delta 2^60
    // 3 delta^2 2^58 = 3 e60^2 / 2^62: with a = |e60| 2^24 (< 2^64), a^2 / 2^64 = e60^2 / 2^16
    const uint64_t a = (uint64_t)(e60 < 0 ? -e60 : e60) << 24;
    const int64_t q = (int64_t)(3ull * (mulhi(a, a) >> 46));
    // z += z (delta/2 + 3 delta^2/8) = z (e60 + q) / 2^61
    const int64_t t = mulhi_s(z, (e60 + q) * 8);      // z (e60 + q) / 2^61
    z = z + (uint64_t)t;
  }
  // S ~ sqrt(t) 2^55 = t z / 2^8 = mt z / 2^60
  uint64_t S = mulhi(mt << 4, z);
  // exact remainder R = mt 2^58 - S^2 (|R| < 2^58), then one fix either way:
  // z is within a few units of 2^63/sqrt(t) (relative 2^-61), so S is off by
  // at most one
  int64_t R = (int64_t)((mt << 58) - S * S);
  if (R < 0) {
    R += (int64_t)(2 * S - 1);
    S -= 1;
  }
  if (R > (int64_t)(2 * S)) {
    R -= (int64_t)(2 * S + 1);
    S += 1;
  }
  // sqrt(x) = sqrt(t) 2^eh = (S + frac) 2^(eh - 55)
  return round_pack(ux & kSgn, S, R != 0, eh);
}

}  // namespace soft
}  // namespace jsvd

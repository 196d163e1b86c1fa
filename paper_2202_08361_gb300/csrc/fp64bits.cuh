// fp64bits.cuh -- exact binary64 exponent manipulation on the integer pipe.
//
// On GB300 the FP64 pipe is narrow, so every operation of the method that
// only moves an exponent or a sign bit (getexp, scalef, abs, copysign, the
// sign "xor" of Alg. d8jac2, the doubling o = 2|a21|) is done here with
// 64-bit integer operations.  All helpers expect finite inputs (the method's
// precondition) and are exact, except ldexp_rn, which rounds to nearest-even
// when the result falls into the subnormal range -- exactly as a single
// IEEE multiplication by 2^k would.
#pragma once
#include <stdint.h>

namespace jsvd {

constexpr uint64_t kSign = 0x8000000000000000ull;
constexpr uint64_t kMant = 0x000FFFFFFFFFFFFFull;
constexpr uint64_t kHidden = 0x0010000000000000ull;
constexpr uint64_t kInf = 0x7FF0000000000000ull;

__device__ __forceinline__ uint64_t bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double dbl(uint64_t u) { return __longlong_as_double((long long)u); }

// floor(lg max(|x|, smallest subnormal)) -- the exponent used by Eq. e:z
// (Listing 1 takes the exponent of max(|x|, DBL_TRUE_MIN), so 0 -> -1074).
__device__ __forceinline__ int flg_sat(double x)
{
  uint64_t a = bits(x) & ~kSign;
  const int e = (int)(a >> 52);
  if (e) return e - 1023;
  a |= (uint64_t)(a == 0);
  return (63 - __clzll((long long)a)) - 1074;
}

// floor(lg |x|) for finite x != 0.
__device__ __forceinline__ int flg(double x) { return flg_sat(x); }

// x * 2^k, rounded to nearest-even; x finite, |k| < 4096.
__device__ __forceinline__ double ldexp_rn(double x, int k)
{
  const uint64_t u = bits(x);
  const uint64_t sign = u & kSign;
  uint64_t a = u & ~kSign;
  if (a == 0) return x;
  int E = (int)(a >> 52);
  uint64_t sig;
  if (E) {
    sig = (a & kMant) | kHidden;
  } else {
    const int lz = __clzll((long long)a) - 11;
    sig = a << lz;
    E = 1 - lz;
  }
  const int E2 = E + k;
  if (E2 >= 2047) return dbl(sign | kInf);
  if (E2 >= 1) return dbl(sign | ((((uint64_t)(E2 - 1)) << 52) + sig));
  const int sh = 1 - E2;
  if (sh >= 54) return dbl(sign);
  uint64_t q = sig >> sh;
  const uint64_t rem = sig & ((1ull << sh) - 1ull);
  const uint64_t half = 1ull << (sh - 1);
  q += (uint64_t)((rem > half) | ((rem == half) & (q & 1ull)));
  return dbl(sign | q);
}

// 2|x| for finite x with |x| <= 2^1022 (exact): shift a subnormal, bump the
// exponent of a normal number.
__device__ __forceinline__ double twice_abs(double x)
{
  const uint64_t a = bits(x) & ~kSign;
  return dbl((a >> 52) ? (a + kHidden) : (a << 1));
}

__device__ __forceinline__ double dabs(double x) { return dbl(bits(x) & ~kSign); }

// |x| with the sign bit of s (copysign)
__device__ __forceinline__ double with_sign(double x, double s)
{
  return dbl((bits(x) & ~kSign) | (bits(s) & kSign));
}

// x with its sign bit XOR-ed with the sign bit of s
__device__ __forceinline__ double xor_sign(double x, double s)
{
  return dbl(bits(x) ^ (bits(s) & kSign));
}

// Order-preserving map of a finite double to int64 (+0 and -0 both -> 0),
// so that x < y  <=>  ord(x) < ord(y), as an IEEE comparison would say.
__device__ __forceinline__ long long ord(double x)
{
  const long long i = __double_as_longlong(x);
  return (i >= 0) ? i : -(i & 0x7FFFFFFFFFFFFFFFll);
}

}  // namespace jsvd

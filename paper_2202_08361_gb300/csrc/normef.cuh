// normef.cuh -- the wide-exponent Frobenius norm of supplement SM6
// (Alg. rnF) for one warp: every lane carries a partial sum of squares as
// r = (e, f) = 2^e f, e an integer (kNegInfE for zero), f in [1, 2), so no
// partial sum overflows or underflows whatever the magnitudes of the
// entries.  Each lane adds its rows in ascending order with the (e, f)
// fma step of SM6.2; the lanes' sums are combined by the (e, f) addition of
// Eq. e:redj in the canonical xor butterfly (16, 8, 4, 2, 1; the addition
// puts the larger operand last, so both lanes of a pair get the same bits);
// the square root of SM6.1 ends it.  Exponents are kept as integers (the
// paper's vector code holds them in floating point); only the fma of each
// step and of each addition runs on the FP64 pipe.
#pragma once
#include <climits>
#include <stdint.h>

#include "fp64bits.cuh"
#include "fp64soft.cuh"

namespace jsvd {

constexpr int kNegInfE = INT_MIN;  // the exponent of zero, -inf

struct EF {
  int e;     // kNegInfE for zero
  double f;  // [1, 2); 1 for zero
};

// getexp / getmant (to [1, 2)) of a finite x; E(0) = -inf, F(0) = 1.
__device__ __forceinline__ int E_of(double x)
{
  return (bits(x) & ~kSign) ? flg(x) : kNegInfE;
}
__device__ __forceinline__ double F_of(double x)
{
  const uint64_t a = bits(x) & ~kSign;
  if (a == 0ull) return 1.0;
  return ldexp_rn(dbl(a), -flg(x));  // exact: a power-of-two scaling into [1, 2)
}

// scalef(f, d) for d <= 0 or d == -inf: f 2^d rounded once (0 for -inf).
__device__ __forceinline__ double scalef_neg(double f, int d)
{
  if (d == kNegInfE) return 0.0;
  return ldexp_rn(f, d < -4000 ? -4000 : d);
}

// r <- fma(|x|, |x|, r) in (e, f) arithmetic (supplement SM6.2).
__device__ __forceinline__ void ef_fma_step(double x, EF &r)
{
  // r' = r with an even (or infinite) exponent
  const int lsb = (r.e == kNegInfE) ? 0 : (r.e & 1);
  const int e1 = (r.e == kNegInfE) ? kNegInfE : r.e - lsb;
  const double f1 = lsb ? twice_abs(r.f) : r.f;  // f in [1, 2): doubling is exact
  const int ex = E_of(x);
  const double fx = F_of(x);
  const int eh = (ex == kNegInfE) ? kNegInfE : 2 * ex;
  const int emax = max(eh, e1);
  const int dh = (eh == kNegInfE) ? kNegInfE : eh - emax;  // even, <= 0
  const int d1 = (e1 == kNegInfE) ? kNegInfE : e1 - emax;
  const double fh = scalef_neg(fx, dh == kNegInfE ? kNegInfE : dh / 2);
  const double fr = scalef_neg(f1, d1);
  const double fn = __fma_rn(fh, fh, fr);
  r.f = F_of(fn);
  r.e = (emax == kNegInfE || (bits(fn) & ~kSign) == 0ull) ? kNegInfE : emax + E_of(fn);
}

// a + b for two (e, f) values (Eq. e:redj: the smaller one scaled by
// 2^(e_small - e_big), then one fma), normalised.  Symmetric in a and b.
__device__ __forceinline__ EF ef_add(EF a, EF b)
{
  const bool a_small = (a.e < b.e) || (a.e == b.e && bits(a.f) <= bits(b.f));
  const EF s = a_small ? a : b, l = a_small ? b : a;
  if (l.e == kNegInfE) return l;  // both zero
  int d = (s.e == kNegInfE) ? INT_MIN : s.e - l.e;
  // 2^d as a double (0 below the subnormal range); d <= 0
  const double t = (d < -1074) ? 0.0 : ldexp_rn(1.0, d);
  const double fn = __fma_rn(t, s.f, l.f);
  EF r;
  r.f = F_of(fn);
  r.e = l.e + E_of(fn);
  return r;
}

__device__ __forceinline__ EF ef_warp_sum(EF r)
{
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    EF q;
    q.e = __shfl_xor_sync(0xffffffffu, r.e, o);
    q.f = __shfl_xor_sync(0xffffffffu, r.f, o);
    r = ef_add(r, q);
  }
  return r;
}

// (e, f) of ||x||^2 -> (e'', f'') of ||x|| (supplement SM6.1); the square
// root on the integer pipe (correctly rounded).
__device__ __forceinline__ EF ef_sqrt(EF r)
{
  if (r.e == kNegInfE) return r;
  EF o;
  double fp = r.f;
  int ep = r.e;
  if (ep & 1) {
    fp = twice_abs(r.f);
    ep -= 1;
  }
  o.e = ep / 2;
  o.f = soft::sqrt_rn(fp);
  return o;
}

}  // namespace jsvd

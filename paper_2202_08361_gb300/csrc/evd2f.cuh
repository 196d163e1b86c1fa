// evd2f.cuh -- the branch-free eigendecomposition of one Hermitian matrix of
// order two in single precision (one thread, one matrix).
//
// Listing 1 (complex) and Alg. d8jac2 (real) with the binary32 constants of
// section 2.4: nu = FLT_MAX, fl(sqrt nu) = 1.844674297E+19, mu =
// FLT_TRUE_MIN, eta = FLT_MAX_EXP - 4 = 124; every operation in binary32
// with round-to-nearest.  Divisions and square roots are the FP32 pipe's
// correctly rounded sequences (__fdiv_rn, __fsqrt_rn); exponent and sign
// manipulations are integer operations on the bit patterns.
#pragma once
#include <stdint.h>

namespace jsvd {

constexpr uint32_t kSignF = 0x80000000u;
constexpr uint32_t kInfF = 0x7F800000u;
constexpr uint32_t kSqrtNuF = 0x5F7FFFFFu;  // fl(sqrt(FLT_MAX)) = 1.844674297E+19

__device__ __forceinline__ uint32_t fbits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float fval(uint32_t u) { return __uint_as_float(u); }

// floor(lg max(|x|, FLT_TRUE_MIN)) (0 -> -149), Eq. e:z's exponent.  Both
// cases are computed and one is selected, so the lanes of a warp never
// diverge (wide-range data mixes normal and subnormal values in a warp).
__device__ __forceinline__ int flgf_sat(float x)
{
  const uint32_t a = fbits(x) & ~kSignF;
  const int e = (int)(a >> 23);
  const int sub = (31 - __clz((int)(a | 1u))) - 149;
  return e ? e - 127 : sub;
}

// x * 2^k rounded to nearest-even (scalbnf); x finite, |k| < 1024.  Branch
// free, like flgf_sat: the normal, subnormal, overflow and zero results are
// all formed and selected.
__device__ __forceinline__ float ldexpf_rn(float x, int k)
{
  const uint32_t u = fbits(x);
  const uint32_t sign = u & kSignF;
  const uint32_t a = u & ~kSignF;
  const int E = (int)(a >> 23);
  const int lz = __clz((int)(a | 1u)) - 8;                 // subnormal normalisation shift
  const uint32_t sig = E ? ((a & 0x007FFFFFu) | 0x00800000u) : (a << (lz > 0 ? lz : 0));
  const int E2 = (E ? E : 1 - lz) + k;
  const uint32_t normal = sign | ((((uint32_t)(E2 - 1)) << 23) + sig);
  int sh = 1 - E2;                                          // right shift into the subnormal grid
  sh = sh < 1 ? 1 : (sh > 25 ? 25 : sh);
  uint32_t q = sig >> sh;
  const uint32_t rem = sig & ((1u << sh) - 1u);
  const uint32_t half = 1u << (sh - 1);
  q += (uint32_t)((rem > half) | ((rem == half) & (q & 1u)));
  uint32_t r = (E2 >= 1) ? normal : (sign | q);
  r = (E2 >= 255) ? (sign | kInfF) : r;
  return fval(a == 0u ? u : r);
}

// a / b, correctly rounded, by the FP32 pipe's fast path.  The operands are
// brought into [1, 2) by exact power-of-two scalings (exponent-field
// rewrites; subnormals are normalised), so the IEEE division's slow path
// (taken near the ends of the exponent range) is never needed; the
// quotient in (1/2, 2) is scaled back by an exponent add, exact in the
// normal range and infinity above it.  A quotient below the normal range
// would be rounded twice that way, so it is redone directly, as are zero,
// infinite and NaN operands.
__device__ __forceinline__ float mant12(float x, int &e)
{
  const uint32_t a = fbits(x) & ~kSignF;
  if (a >= 0x00800000u) {
    e = (int)(a >> 23) - 127;
    return fval((fbits(x) & 0x807FFFFFu) | 0x3F800000u);
  }
  const int lz = __clz((int)a) - 8;  // subnormal: shift the leading bit into place
  e = -126 - lz;
  return fval((fbits(x) & kSignF) | 0x3F800000u | ((a << lz) & 0x007FFFFFu));
}

__device__ __forceinline__ float div_fast(float a, float b)
{
  const uint32_t ua = fbits(a) & ~kSignF, ub = fbits(b) & ~kSignF;
  if (ua == 0u || ub == 0u || ua >= kInfF || ub >= kInfF) return __fdiv_rn(a, b);
  int ea, eb;
  const float q = __fdiv_rn(mant12(a, ea), mant12(b, eb));  // |q| in (1/2, 2)
  const int k = ea - eb;
  const int eq = (int)((fbits(q) >> 23) & 0xFFu) + k;  // biased exponent of the result
  if (eq <= 0) return __fdiv_rn(a, b);
  if (eq >= 255) return fval((fbits(q) & kSignF) | kInfF);
  return fval(fbits(q) + ((uint32_t)k << 23));
}

// sqrt(x), correctly rounded, x >= 0 finite: x = m 2^(2j), m in [1, 4)
// (exact), sqrt(m) in [1, 2) by the fast path, then 2^j added exactly.
__device__ __forceinline__ float sqrt_fast(float x)
{
  const uint32_t a = fbits(x) & ~kSignF;
  if (a == 0u || a >= kInfF) return __fsqrt_rn(x);
  int e;
  float m = mant12(x, e);
  if (e & 1) {  // make the exponent even: m in [2, 4)
    m = fval(fbits(m) + 0x00800000u);
    e -= 1;
  }
  const float r = __fsqrt_rn(m);
  return fval(fbits(r) + ((uint32_t)(e / 2) << 23));
}

template <bool FAST>
__device__ __forceinline__ float fdiv(float a, float b)
{
  if constexpr (FAST) return div_fast(a, b);
  else return __fdiv_rn(a, b);
}

template <bool FAST>
__device__ __forceinline__ float fsqrt(float x)
{
  if constexpr (FAST) return sqrt_fast(x);
  else return __fsqrt_rn(x);
}

struct Rot2f {
  float cphi, etr, eti, l1s, l2s;
  int zeta;
};

// Section 2.1 from the scaled a11', a22' and |a21'|.
template <bool FAST>
__device__ __forceinline__ void rot_core_f(float a11, float a22, float aa21, float &tan1,
                                          float &sec2, float &o, float &cphi)
{
  o = __fmul_rn(aa21, 2.0f);  // exact
  const float a = __fsub_rn(a11, a22);
  // Eq. e:tan2: min(max(o/|a|, 0), fl(sqrt nu)) with the sign of a (0/0 -> 0)
  const float q = fmaxf(fdiv<FAST>(o, fabsf(a)), 0.0f);
  const float tan2 = copysignf(fminf(q, fval(kSqrtNuF)), a);
  tan1 = fdiv<FAST>(tan2, __fadd_rn(1.0f, fsqrt<FAST>(__fmaf_rn(tan2, tan2, 1.0f))));
  sec2 = __fmaf_rn(tan1, tan1, 1.0f);
  cphi = fdiv<FAST>(1.0f, fsqrt<FAST>(sec2));
}

template <bool FAST>
__device__ __forceinline__ void lambdas_f(Rot2f &r, float a11, float a22, float tan1, float sec2,
                                          float o)
{
  r.l1s = fdiv<FAST>(__fmaf_rn(tan1, __fmaf_rn(a22, tan1, o), a11), sec2);
  r.l2s = fdiv<FAST>(__fmaf_rn(tan1, __fmaf_rn(a11, tan1, -o), a22), sec2);
}

// Real symmetric (Alg. d8jac2 in binary32).
template <bool FAST>
__device__ __forceinline__ Rot2f ssjac2(float a11, float a22, float a21)
{
  Rot2f r;
  r.zeta = 124 - max(max(flgf_sat(a11), flgf_sat(a22)), flgf_sat(a21));
  a11 = ldexpf_rn(a11, r.zeta);
  a22 = ldexpf_rn(a22, r.zeta);
  a21 = ldexpf_rn(a21, r.zeta);
  float tan1, sec2, o;
  rot_core_f<FAST>(a11, a22, fabsf(a21), tan1, sec2, o, r.cphi);
  r.etr = fval(fbits(tan1) ^ (fbits(a21) & kSignF));
  r.eti = 0.0f;
  lambdas_f<FAST>(r, a11, a22, tan1, sec2, o);
  return r;
}

// Complex Hermitian (Listing 1 in binary32).
template <bool FAST>
__device__ __forceinline__ Rot2f csjac2(float a11, float a22, float a21r, float a21i)
{
  Rot2f r;
  r.zeta = 124 - max(max(flgf_sat(a11), flgf_sat(a22)), max(flgf_sat(a21r), flgf_sat(a21i)));
  a11 = ldexpf_rn(a11, r.zeta);
  a22 = ldexpf_rn(a22, r.zeta);
  a21r = ldexpf_rn(a21r, r.zeta);
  a21i = ldexpf_rn(a21i, r.zeta);
  const float ar = fabsf(a21r), ai = fabsf(a21i);
  const float am = fminf(ar, ai), aM = fmaxf(ar, ai);
  const float mM = fmaxf(fdiv<FAST>(am, aM), 0.0f);  // 0/0 -> 0
  const float aa21 = __fmul_rn(fsqrt<FAST>(__fmaf_rn(mM, mM, 1.0f)), aM);
  const float ca = copysignf(fminf(fdiv<FAST>(ar, aa21), 1.0f), a21r);
  const float sa = fdiv<FAST>(a21i, fmaxf(aa21, fval(1u)));  // fval(1) = FLT_TRUE_MIN
  float tan1, sec2, o;
  rot_core_f<FAST>(a11, a22, aa21, tan1, sec2, o, r.cphi);
  r.etr = __fmul_rn(ca, tan1);
  r.eti = __fmul_rn(sa, tan1);
  lambdas_f<FAST>(r, a11, a22, tan1, sec2, o);
  return r;
}

__device__ __forceinline__ int32_t pack_zp_f(const Rot2f &r)
{
  return (int32_t)((((uint32_t)(-r.zeta)) << 1) | (uint32_t)(r.l1s < r.l2s));
}

}  // namespace jsvd

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

// x 2^z for the prescaling of Eq. e:z, z = eta - floor(lg max|a_ij|) in
// [-3, 273], by three multiplications by powers of two on the FP32 pipe:
// 2^min(z, 127), then the rest of z in at most two factors >= 1.  Only the
// first can round (z < 0, a result below the normal range: one rounding,
// as ldexpf_rn); every later one scales up a value that stays below
// 2^125, which is exact.
__device__ __forceinline__ float scale_zeta(float x, int z)
{
  const int z1 = min(z, 127), z2 = min(max(z - 127, 0), 127), z3 = max(z - 254, 0);
  const float p1 = fval((uint32_t)(z1 + 127) << 23);
  const float p2 = fval((uint32_t)(z2 + 127) << 23);
  const float p3 = fval((uint32_t)(z3 + 127) << 23);
  return __fmul_rn(__fmul_rn(__fmul_rn(x, p1), p2), p3);
}

// floor(lg max(|x|, |y|, |w|, |v|, FLT_TRUE_MIN)): the larger magnitude has
// the larger bit pattern, so one exponent extraction serves all.
__device__ __forceinline__ int flgf_max(float x, float y, float w, float v)
{
  const uint32_t m = max(max(fbits(x) & ~kSignF, fbits(y) & ~kSignF),
                         max(fbits(w) & ~kSignF, fbits(v) & ~kSignF));
  return flgf_sat(fval(m));
}

// The significand of |x| (bits a, a != 0) scaled into [1, 2) and its
// exponent: x = m 2^e exactly; subnormals are normalised.  Both forms are
// computed and one selected, so the lanes of a warp never diverge.
__device__ __forceinline__ float norm12(uint32_t a, int &e)
{
  const int E = (int)(a >> 23);
  const int p = 31 - __clz((int)(a | 1u));                 // top set bit of a subnormal
  const uint32_t msub = (a << ((23 - p) & 31)) & 0x007FFFFFu;
  e = E ? E - 127 : p - 149;
  return fval(0x3F800000u | (E ? (a & 0x007FFFFFu) : msub));
}

// a / b, correctly rounded (to nearest-even), for finite a and b (b = 0
// gives IEEE's Inf or NaN), without a data-dependent branch: the operands are scaled into
// [1, 2) (exactly), their quotient q in (1/2, 2) is taken by the IEEE
// division (which never needs its slow path there) together with the exact
// remainder r = a' - q b' (one fma), and the result is rebuilt from q's
// significand and the exponent difference.  A result below the normal range
// is rounded once more on the subnormal grid: the bits of q shifted out
// decide, except when they are exactly half an ulp of that grid, where q
// sits on the midpoint itself and the sign of r tells on which side of it
// the exact quotient lies (r = 0: a tie, to even).  The midpoint is a
// 24-bit number, so q (the correctly rounded quotient) is below, on or above
// it exactly when the exact quotient is.
__device__ __forceinline__ float div_fast(float a, float b)
{
  const uint32_t ua = fbits(a), ub = fbits(b);
  const uint32_t sign = (ua ^ ub) & kSignF;
  const uint32_t xa = ua & ~kSignF, xb = ub & ~kSignF;
  int ea, eb;
  const float ma = norm12(xa, ea), mb = norm12(xb, eb);
  const float q = __fdiv_rn(ma, mb);
  const float r = __fmaf_rn(-q, mb, ma);  // exact
  const uint32_t uq = fbits(q);
  const int E = ea - eb + (int)(uq >> 23) - 127;           // exponent of the result
  const uint32_t sig = (uq & 0x007FFFFFu) | 0x00800000u;  // q's 24-bit significand
  const uint32_t normal = (((uint32_t)(E + 127)) << 23) | (sig & 0x007FFFFFu);
  int sh = -126 - E;                                      // right shift onto the grid 2^-149
  sh = sh < 1 ? 1 : (sh > 25 ? 25 : sh);
  uint32_t qs = sig >> sh;
  const uint32_t lost = sig & ((1u << sh) - 1u), half = 1u << (sh - 1);
  const uint32_t rb = fbits(r);
  const bool r_pos = (rb & ~kSignF) != 0u && !(rb & kSignF);
  const bool r_zero = (rb & ~kSignF) == 0u;
  qs += (uint32_t)((lost > half) | ((lost == half) & (r_pos | (r_zero & ((qs & 1u) != 0u)))));
  uint32_t res = (E >= -126) ? normal : qs;
  res = (E > 127) ? kInfF : res;
  res = (xa == 0u) ? 0u : res;
  // a zero divisor gives what IEEE division gives (the EVD's clamps rely on
  // it): Inf, or NaN for 0/0
  res = (xb == 0u) ? ((xa == 0u) ? 0x7FC00000u : kInfF) : res;
  return fval(sign | res);
}

// Which division each site takes: bit SITE of DM set, the branch-free
// div_fast; clear, the IEEE division.  Sites:
//   0 o/|a|   1 tan(phi)   2 1/sec(phi)   3 lambda1'   4 lambda2'
//   5 am/aM   6 |Re a21'|/|a21'|   7 Im a21'/|a21'|
// On wide-range data the quotients of sites 0, 1, 5, 6 and 7 leave the
// normal range in 4 - 30 % of the lanes, so that nearly every warp would run
// the IEEE slow path there; those of 2 - 4 almost never.  Both round
// correctly, so DM changes no bit.
template <int DM, int SITE>
__device__ __forceinline__ float fdiv(float a, float b)
{
  if constexpr (((DM >> SITE) & 1) != 0) return div_fast(a, b);
  else return __fdiv_rn(a, b);
}

// The EVD's square roots all take operands in [1, fl(sqrt nu)^2 + 1]
// (x^2 + 1, sec^2), where the IEEE routine never leaves its fast path.
__device__ __forceinline__ float fsqrt(float x) { return __fsqrt_rn(x); }

struct Rot2f {
  float cphi, etr, eti, l1s, l2s;
  int zeta;
};

// Section 2.1 from the scaled a11', a22' and |a21'|.
template <int DM>
__device__ __forceinline__ void rot_core_f(float a11, float a22, float aa21, float &tan1,
                                          float &sec2, float &o, float &cphi)
{
  o = __fmul_rn(aa21, 2.0f);  // exact
  const float a = __fsub_rn(a11, a22);
  // Eq. e:tan2: min(max(o/|a|, 0), fl(sqrt nu)) with the sign of a (0/0 -> 0)
  const float q = fmaxf(fdiv<DM, 0>(o, fabsf(a)), 0.0f);
  const float tan2 = copysignf(fminf(q, fval(kSqrtNuF)), a);
  tan1 = fdiv<DM, 1>(tan2, __fadd_rn(1.0f, fsqrt(__fmaf_rn(tan2, tan2, 1.0f))));
  sec2 = __fmaf_rn(tan1, tan1, 1.0f);
  cphi = fdiv<DM, 2>(1.0f, fsqrt(sec2));
}

template <int DM>
__device__ __forceinline__ void lambdas_f(Rot2f &r, float a11, float a22, float tan1, float sec2,
                                          float o)
{
  r.l1s = fdiv<DM, 3>(__fmaf_rn(tan1, __fmaf_rn(a22, tan1, o), a11), sec2);
  r.l2s = fdiv<DM, 4>(__fmaf_rn(tan1, __fmaf_rn(a11, tan1, -o), a22), sec2);
}

// Real symmetric (Alg. d8jac2 in binary32).
template <int DM>
__device__ __forceinline__ Rot2f ssjac2(float a11, float a22, float a21)
{
  Rot2f r;
  r.zeta = 124 - flgf_max(a11, a22, a21, 0.0f);
  a11 = scale_zeta(a11, r.zeta);
  a22 = scale_zeta(a22, r.zeta);
  a21 = scale_zeta(a21, r.zeta);
  float tan1, sec2, o;
  rot_core_f<DM>(a11, a22, fabsf(a21), tan1, sec2, o, r.cphi);
  r.etr = fval(fbits(tan1) ^ (fbits(a21) & kSignF));
  r.eti = 0.0f;
  lambdas_f<DM>(r, a11, a22, tan1, sec2, o);
  return r;
}

// Complex Hermitian (Listing 1 in binary32).
template <int DM>
__device__ __forceinline__ Rot2f csjac2(float a11, float a22, float a21r, float a21i)
{
  Rot2f r;
  r.zeta = 124 - flgf_max(a11, a22, a21r, a21i);
  a11 = scale_zeta(a11, r.zeta);
  a22 = scale_zeta(a22, r.zeta);
  a21r = scale_zeta(a21r, r.zeta);
  a21i = scale_zeta(a21i, r.zeta);
  const float ar = fabsf(a21r), ai = fabsf(a21i);
  const float am = fminf(ar, ai), aM = fmaxf(ar, ai);
  const float mM = fmaxf(fdiv<DM, 5>(am, aM), 0.0f);  // 0/0 -> 0
  const float aa21 = __fmul_rn(fsqrt(__fmaf_rn(mM, mM, 1.0f)), aM);
  const float ca = copysignf(fminf(fdiv<DM, 6>(ar, aa21), 1.0f), a21r);
  const float sa = fdiv<DM, 7>(a21i, fmaxf(aa21, fval(1u)));  // fval(1) = FLT_TRUE_MIN
  float tan1, sec2, o;
  rot_core_f<DM>(a11, a22, aa21, tan1, sec2, o, r.cphi);
  r.etr = __fmul_rn(ca, tan1);
  r.eti = __fmul_rn(sa, tan1);
  lambdas_f<DM>(r, a11, a22, tan1, sec2, o);
  return r;
}

__device__ __forceinline__ int32_t pack_zp_f(const Rot2f &r)
{
  return (int32_t)((((uint32_t)(-r.zeta)) << 1) | (uint32_t)(r.l1s < r.l2s));
}

}  // namespace jsvd

// evd2.cuh -- the branch-free eigendecomposition of one Hermitian matrix of
// order two, as a device function (one thread, one matrix).
//
// It computes what Listing 1 (complex) and Alg. d8jac2 (real, supplement
// SM2.1) of the paper compute, operation for operation in binary64 with
// round-to-nearest: the prescaling exponent of Eq. e:z, the polar form of
// Eq. e:zpolar with the naive hypot of Alg. hypot, tan(2 phi) clamped as in
// Eq. e:tan2, tan(phi) from Eq. e:jactan, sec^2, sec and cos(phi) from
// Eq. e:jacsec (never rsqrt), the eigenvalues of Eq. e:lamsec and the
// permutation bit p = (lambda1' < lambda2').  Exponent and sign
// manipulations run on the integer pipe (fp64bits.cuh); the IEEE
// min/max filtering of NaN becomes explicit integer selects that give the
// same result for the only NaNs that can arise (0/0).
#pragma once
#include "fp64bits.cuh"
#include "fp64soft.cuh"

namespace jsvd {

// fl(sqrt(nu)) of Eq. e:tan2: the largest double whose square is below
// DBL_MAX; as a bit pattern.
constexpr uint64_t kSqrtNuBits = 0x5FEFFFFFFFFFFFFFull;

// Eq. e:tan2 after the division: q = o/|a| in [0, +inf] or NaN (0/0).
// Returns min(fmax(q, 0), fl(sqrt nu)) with the sign of a.
__device__ __forceinline__ double clamp_tan2(double q, double a)
{
  uint64_t qb = bits(q);
  qb = (qb > kInf) ? 0ull : qb;                   // fmax(NaN, 0) = 0
  qb = (qb > kSqrtNuBits) ? kSqrtNuBits : qb;     // fmin(., fl(sqrt nu))
  return dbl(qb | (bits(a) & kSign));
}

// floor(lg max(|x|, |y|, |w|, |v|, DBL_TRUE_MIN)) of Eq. e:z: the larger
// magnitude has the larger bit pattern, so one exponent extraction serves
// all four.
__device__ __forceinline__ int flg_max(double x, double y, double w, double v)
{
  const uint64_t m = max(max(bits(x) & ~kSign, bits(y) & ~kSign), max(bits(w) & ~kSign, bits(v) & ~kSign));
  return flg_sat(dbl(m));
}

struct Rot2 {
  double cphi;   // cos(phi)
  double etr;    // Re(e^{i alpha} tan(phi)) (real: sign(a21) tan(phi))
  double eti;    // Im(e^{i alpha} tan(phi)) (real: 0)
  double l1s;    // lambda1' (scaled)
  double l2s;    // lambda2' (scaled)
  int zeta;      // Eq. e:z exponent
};

// Where each division and square root runs.  Bit SLOT of MASK set: the
// integer-pipe routine of fp64soft.cuh; clear: the FP64 pipe's IEEE
// instruction.  Both are correctly rounded, so every MASK gives the same
// bits; the choice only balances the two pipes.  Slots:
//   0 o/|a|   1 sqrt(tan2^2 + 1)   2 tan2/(1 + sqrt)   3 sqrt(sec^2)
//   4 1/sec   5 lambda1' / sec^2   6 lambda2' / sec^2
//   7 am/aM   8 sqrt(mM^2 + 1)     9 |Re a21'|/|a21'|  10 Im a21'/|a21'|
template <int MASK, int SLOT>
__device__ __forceinline__ double dv(double a, double b)
{
  if constexpr (((MASK >> SLOT) & 1) != 0) return soft::div_rn(a, b);
  else return __ddiv_rn(a, b);
}

template <int MASK, int SLOT>
__device__ __forceinline__ double sq(double x)
{
  if constexpr (((MASK >> SLOT) & 1) != 0) return soft::sqrt_rn(x);
  else return __dsqrt_rn(x);
}

// The rotation part shared by the real and the complex case, from the
// scaled a11', a22' and |a21'| (section 2.1).
template <int MASK>
__device__ __forceinline__ void rot_core(double a11, double a22, double aa21, double &tan1,
                                         double &sec2, double &o, double &cphi)
{
  o = twice_abs(aa21);                          // o = 2|a21'|, exact
  const double a = __dsub_rn(a11, a22);
  // Eq. e:tan2; |a| = 0 gives o/|a| = Inf (o > 0) or NaN (o = 0), which the
  // clamp turns into fl(sqrt nu) or 0 -- selected here without dividing
  const double aa = dabs(a);
  const double q = (bits(aa) == 0ull) ? ((bits(o) == 0ull) ? 0.0 : dbl(kInf)) : dv<MASK, 0>(o, aa);
  const double tan2 = clamp_tan2(q, a);
  tan1 = dv<MASK, 2>(tan2, __dadd_rn(1.0, sq<MASK, 1>(__fma_rn(tan2, tan2, 1.0))));
  sec2 = __fma_rn(tan1, tan1, 1.0);
  cphi = dv<MASK, 4>(1.0, sq<MASK, 3>(sec2));
}

// Eq. e:lamsec: lambda1' and lambda2' (scaled).  When both divisions run on
// the integer pipe they share the prepared divisor sec^2.
template <int MASK>
__device__ __forceinline__ void lambdas(Rot2 &r, double a11, double a22, double tan1, double sec2,
                                        double o)
{
  const double n1 = __fma_rn(tan1, __fma_rn(a22, tan1, o), a11);
  const double n2 = __fma_rn(tan1, __fma_rn(a11, tan1, -o), a22);
  if constexpr (((MASK >> 5) & 1) != 0 && ((MASK >> 6) & 1) != 0) {
    const soft::Den D = soft::prepare_den(sec2);
    r.l1s = soft::div_rn(n1, D);
    r.l2s = soft::div_rn(n2, D);
  } else {
    r.l1s = dv<MASK, 5>(n1, sec2);
    r.l2s = dv<MASK, 6>(n2, sec2);
  }
}

// Real symmetric matrix (Alg. d8jac2).
template <int MASK>
__device__ __forceinline__ Rot2 dsjac2(double a11, double a22, double a21)
{
  Rot2 r;
  r.zeta = 1020 - flg_max(a11, a22, a21, 0.0);  // eta - floor(lg max|a_ij|), eta = 1020
  a11 = ldexp_rn(a11, r.zeta);
  a22 = ldexp_rn(a22, r.zeta);
  a21 = ldexp_rn(a21, r.zeta);
  double tan1, sec2, o;
  rot_core<MASK>(a11, a22, dabs(a21), tan1, sec2, o, r.cphi);
  r.etr = xor_sign(tan1, a21);
  r.eti = 0.0;
  lambdas<MASK>(r, a11, a22, tan1, sec2, o);
  return r;
}

// Complex Hermitian matrix (Listing 1).
template <int MASK>
__device__ __forceinline__ Rot2 zsjac2(double a11, double a22, double a21r, double a21i)
{
  Rot2 r;
  r.zeta = 1020 - flg_max(a11, a22, a21r, a21i);
  a11 = ldexp_rn(a11, r.zeta);
  a22 = ldexp_rn(a22, r.zeta);
  a21r = ldexp_rn(a21r, r.zeta);
  a21i = ldexp_rn(a21i, r.zeta);
  // polar form of a21' (Eq. e:zpolar), |a21'| by Alg. hypot
  const double ar = dabs(a21r), ai = dabs(a21i);
  const bool rmin = bits(ar) <= bits(ai);
  const double am = rmin ? ar : ai, aM = rmin ? ai : ar;
  const bool zero = (bits(aM) == 0ull);
  const double mM = zero ? 0.0 : dv<MASK, 7>(am, aM);              // fmax(am/aM, 0)
  const double aa21 = __dmul_rn(sq<MASK, 8>(__fma_rn(mM, mM, 1.0)), aM);
  double qc, qs;  // |Re a21'| / |a21'| and Im a21' / |a21'|
  if constexpr (((MASK >> 9) & 1) != 0 && ((MASK >> 10) & 1) != 0) {
    const soft::Den D = soft::prepare_den(aa21);  // one divisor, prepared once
    qc = soft::div_rn(ar, D);
    qs = soft::div_rn(a21i, D);
  } else {
    qc = dv<MASK, 9>(ar, aa21);
    qs = dv<MASK, 10>(a21i, aa21);
  }
  const double ca = with_sign(zero ? 1.0 : qc, a21r);  // fmin(., 1)
  const double sa = zero ? a21i : qs;                  // / fmax(|a21|, mu)
  double tan1, sec2, o;
  rot_core<MASK>(a11, a22, aa21, tan1, sec2, o, r.cphi);
  r.etr = __dmul_rn(ca, tan1);
  r.eti = __dmul_rn(sa, tan1);
  lambdas<MASK>(r, a11, a22, tan1, sec2, o);
  return r;
}

// The division placement used inside the SVD kernels, where the FP64 pipe
// is busy with the column work: everything on the integer pipe.
constexpr int kMaskAllSoft = 0x7FF;

// p = (lambda1' < lambda2'), as an IEEE comparison (lambda' finite).
__device__ __forceinline__ int perm_bit(const Rot2 &r) { return ord(r.l1s) < ord(r.l2s); }

// (zeta' << 1) | p with zeta' = -zeta, formed by an unsigned shift.
__device__ __forceinline__ int32_t pack_zp(const Rot2 &r)
{
  return (int32_t)((((uint32_t)(-r.zeta)) << 1) | (uint32_t)perm_bit(r));
}

}  // namespace jsvd

// svd_core.cuh -- one warp, one pivot pair: the fused step of the one-sided
// Jacobi SVD (Alg. zvjsvd, lines spade..star), shared by the single-matrix
// persistent kernel and the batched kernel.
//
// The warp reads the pair's columns once for the three sums, reduces them
// in a canonical order (lane l accumulates rows l, l+32, l+64, ... in
// ascending order with fma, then one fixed reduction tree over the lanes for
// all the sums, warp_sum_slots), so the bits never depend on the launch
// shape.  Lane 0 forms the (e,f)
// norms, the scaled dot-product (Alg. zdpscl semantics: power-of-two
// prescaling, one final division by f_q f_p), the convergence test
// (Eq. e:tol, Alg. cvg), the scaled Grammian (Alg. Gram) and its 2x2 EVD,
// and broadcasts the rotation; the whole warp then applies Eq. e:transf
// (Alg. zjrot) to the G and V column pairs, swapping per the permutation
// bit, and tracks the max-norm of the new G columns (section 3.2, step 4).
#pragma once
#include <climits>

#include "evd2.cuh"
#include "fp64sel.cuh"
#include "normef.cuh"

namespace jsvd {

// Loads and stores of G and V inside the persistent kernels bypass L1: a
// column written by another SM in the previous step must not be served from
// a stale L1 line (L1 is not coherent across SMs; the grid barrier only
// orders L2).
__device__ __forceinline__ double ldg2(const double *p) { return __ldcg(p); }
__device__ __forceinline__ void stg2(double *p, double v) { __stcg(p, v); }
__device__ __forceinline__ float ldg2(const float *p) { return __ldcg(p); }
__device__ __forceinline__ void stg2(float *p, float v) { __stcg(p, v); }

// One rounding per operation in the column precision T.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double mul_t(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_t(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double to_t(double x, double) { return x; }
__device__ __forceinline__ float to_t(double x, float) { return __double2float_rn(x); }

// Magnitude bits of a finite value, widened so that the order of the
// magnitudes is the order of the integers; magbits_to_double inverts it.
__device__ __forceinline__ unsigned long long magbits(double x)
{
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long magbits(float x)
{
  return (unsigned long long)((unsigned)__float_as_int(x) & 0x7FFFFFFFu);
}
__device__ __forceinline__ double magbits_to_double(unsigned long long b, double)
{
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double magbits_to_double(unsigned long long b, float)
{
  return (double)__int_as_float((int)(unsigned)b);  // exact widening
}

// How the kernels reach the iteration matrix's columns.
constexpr int kAccPlain = 0;  // plain loads and stores: one block owns the matrix (in
                              // global or in shared memory); block barriers order the
                              // accesses and L1 may serve them
constexpr int kAccL2 = 1;     // through L2 only (ldg2/stg2): blocks on several SMs
                              // update the matrix

// The iteration matrix G (m x n) and V (n x n) in column precision T.
template <typename T, int CG = kAccL2>
struct MatViewT {
  T *gr, *gi;        // G planes (gi == nullptr for real), column j at Gr(j)
  T *vr, *vi;        // V planes, column j at Vr(j)
  int m, n;          // true sizes
  int mp, np;        // rows padded to a multiple of 32 (padding rows are 0)
  int64_t ldg, ldv;

  __device__ __forceinline__ T *Gr(int j) const { return gr + j * ldg; }
  __device__ __forceinline__ T *Gi(int j) const { return gi + j * ldg; }
  __device__ __forceinline__ T *Vr(int j) const { return vr + j * ldv; }
  __device__ __forceinline__ T *Vi(int j) const { return vi + j * ldv; }

  static __device__ __forceinline__ T ld(const T *p)
  {
    if constexpr (CG == kAccL2) return ldg2(p);
    else return *p;
  }
  static __device__ __forceinline__ void st(T *p, T v)
  {
    if constexpr (CG == kAccL2) stg2(p, v);
    else *p = v;
  }
};
using MatView = MatViewT<double>;

// The binade the iteration matrix's max-norm is brought to, at the start
// and by every rescaling (section 3.2), for the rescale bound 2^rexp: 24
// binades below the bound (no rescaling while the max-norm grows by less
// than 2^24, about sqrt(m n) at most), 0 for small bounds.  The high scale
// leaves tiny columns the most room above the subnormal range; the squares
// of an m x n G below 2^480 cannot overflow for m <= 2^24.
__host__ __device__ __forceinline__ int scale_target(int rexp) { return rexp > 25 ? rexp - 25 : 0; }

// The round-robin parallel ordering (section 4.1): pair l of step k among
// nt (even) columns; pairs with q >= n are phantom pairs.
__device__ __forceinline__ void pair_of(int k, int l, int nt, int &p, int &q)
{
  const int K = nt - 1;
  if (l == 0) {
    p = k;
    q = nt - 1;
    return;
  }
  int a = k + l;
  if (a >= K) a -= K;
  int b = k - l;
  if (b < 0) b += K;
  p = min(a, b);
  q = max(a, b);
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
  for (int o = 16; o; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Sums over the warp of N per-lane values (N = 4 or 16) in a fixed tree
// that spends 6 (N = 4) or 16 (N = 16) FP64 additions per lane instead of
// the 5 N of one butterfly per value: at the
// stages with offsets 16, 8, ... the two lanes of a pair split the values
// still held (the lane with the offset bit clear keeps the lower half) and
// each adds its partner's copies of the half it keeps; once one value is
// left the remaining offsets are a plain xor butterfly.  On return lane l
// holds the total of slot (l >> (5 - lg N)) in v[0]; warp_slot() reads a
// slot from any lane.  The tree does not depend on the launch.
template <int N>
__device__ __forceinline__ double warp_sum_slots(double (&v)[N])
{
  static_assert(N == 4 || N == 16, "4 or 16 slots");
  const int lane = threadIdx.x & 31;
  int count = N;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    if (count > 1) {
      const int half = count / 2;
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int k = 0; k < N / 2; ++k) {
        if (k < half) {
          const double keep = up ? v[k + half] : v[k];
          const double send = up ? v[k] : v[k + half];
          v[k] = __dadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
      }
      count = half;
    } else {
      v[0] = __dadd_rn(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
    }
  }
  return v[0];
}

// Slot k of a warp_sum_slots<N> result, broadcast to every lane.
template <int N>
__device__ __forceinline__ double warp_slot(double x, int k)
{
  return __shfl_sync(0xffffffffu, x, k * (32 / N));
}

// Max over the warp of a 64-bit unsigned value (all lanes active): the
// largest upper half by one redux.sync, then the largest lower half among
// the lanes that hold it.
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long x)
{
  const unsigned int hi = (unsigned int)(x >> 32);
  const unsigned int mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned int ml = __reduce_max_sync(0xffffffffu, (hi == mh) ? (unsigned int)x : 0u);
  return ((unsigned long long)mh << 32) | ml;
}

// |x| bits of a finite double: ordered like the magnitudes
__device__ __forceinline__ unsigned long long abits(double x) { return bits(x) & ~kSign; }

// Alg. hypot (naive, reproducible)
__device__ __forceinline__ double hypot_naive(double x, double y)
{
  const double ax = dabs(x), ay = dabs(y);
  const bool xm = bits(ax) <= bits(ay);
  const double m = xm ? ax : ay, M = xm ? ay : ax;
  const double q = (bits(M) == 0ull) ? 0.0 : soft::div_rn(m, M);
  return __dmul_rn(soft::sqrt_rn(__fma_rn(q, q, 1.0)), M);
}

// x 2^k for the FP32 phase (never used with k != 0 there: that phase does
// not rescale; scalbnf is exact unless the result leaves the normal range).
__device__ __forceinline__ float ldexp_rn(float x, int k) { return scalbnf(x, k); }

// Scale a column by 2^k in place (rows < mp).
template <typename T, int CG>
__device__ __forceinline__ void scale_col(const MatViewT<T, CG> &M, T *x, int k, int lane)
{
  for (int i = lane; i < M.mp; i += 32) M.st(x + i, ldexp_rn(M.ld(x + i), k));
}

struct PairOut {
  bool rot, swap;
  double c, C, S;
  // Gram-Schmidt step (Eq. e:GS) in place of the rotation on G: gs = 1
  // orthogonalises g_q against g_p, gs = 2 g_p against g_q; the source
  // column is scaled by 2^-ex, the target by 2^-ey, psi = (psr + i psi) psq
  // (the product is formed by gs_apply, off the rotation's path)
  int gs, ex, ey;
  double psr, psi, psq;
};

// Eq. e:GScond in (e, f) form: ||x|| > 2^eta^ upsilon ||y||, eta^ = 1023,
// with q = fx / fy already formed: fl(q 2^d) > upsilon, d = ex - ey - 1023
// (clamped).  q = f_p / f_q or f_q / f_p lies in [1/2, 2] (f in [1, 2)) and
// upsilon = 2^-53 sqrt(m) (2^-20 sqrt(m) in the FP32 phase) is normal, so
// the comparison needs no rounding (soft::gt_scaled_pos).
__device__ __forceinline__ bool gs_cond(int ex, int ey, double q, double ups)
{
  int d = ex - ey - 1023;
  d = d > 4000 ? 4000 : (d < -4000 ? -4000 : d);
  return soft::gt_scaled_pos(q, d, ups);
}

// Section 3.5.1: for a pair to be rotated whose norms are this far apart,
// Eq. e:GS replaces the rotation of G (Alg. zvjsvd checks Eq. e:GScond
// before zjrot); V still takes the rotation.  gs = 1 orthogonalises g_q
// against g_p (psi = conj(a21') f_q / f_p), gs = 2 g_p against g_q
// (psi = a21' f_p / f_q).  Selects only, so that the compiler may place it
// beside the rotation's chain; o's Gram-Schmidt fields are 0 when gs = 0.
__device__ __forceinline__ void gs_select(PairOut &o, int ep, int eq, double q12, double q21,
                                          double zr, double zi, double ups)
{
  const bool c1 = gs_cond(ep, eq, q12, ups), c2 = gs_cond(eq, ep, q21, ups);
  const int gs = !o.rot ? 0 : c1 ? 1 : c2 ? 2 : 0;
  o.gs = gs;
  o.ex = (gs == 1) ? ep : (gs == 2) ? eq : 0;
  o.ey = (gs == 1) ? eq : (gs == 2) ? ep : 0;
  o.psr = gs ? zr : 0.0;
  o.psi = (gs == 1) ? dbl(bits(zi) ^ kSign) : (gs == 2) ? zi : 0.0;  // conj(a21') for gs = 1
  o.psq = (gs == 1) ? q21 : (gs == 2) ? q12 : 0.0;
}


// The sums of one pivot pair.  Normally pp = ||g_p||^2, qq = ||g_q||^2 and
// (qr, qi) = g_q^* g_p of the current G.  When a column's squares underflow
// (wide): (ep, fp), (eq, fq) are the columns' norms from Alg. rnF and
// (qr, qi) = (g_q / 2^eq)^* (g_p / 2^ep), the prescaled dot-product of
// Alg. zdpscl.
struct PairSums {
  double pp, qq, qr, qi;
  double fp, fq;
  int ep, eq;
  int wide;
};

// From the sums to the rotation (Alg. zdpscl's division, Alg. cvg,
// Alg. Gram, the EVD); its divisions and square roots run on the integer
// pipe (fp64soft.cuh, correctly rounded), leaving the FP64 pipe to the
// column work.  spp = ||g_p||^2, sqq = ||g_q||^2,
// (sqr, sqi) = g_q^* g_p, all of the current (scaled) G.
template <bool CPLX>
__device__ __forceinline__ PairOut pair_rotation(const PairSums &sm, double ups)
{
  PairOut o;
  o.c = 1.0;
  o.C = 0.0;
  o.S = 0.0;
  o.gs = 0;
  o.ex = o.ey = 0;
  o.psr = o.psi = o.psq = 0.0;
  int ep, eq, shift;
  double fp, fq;
  if (sm.wide) {
    // norms from Alg. rnF; the dot-product is already prescaled
    if (sm.ep == kNegInfE || sm.eq == kNegInfE) {
      o.rot = false;
      o.swap = (sm.ep == kNegInfE) && (sm.eq != kNegInfE);  // ||g_p|| < ||g_q||
      return o;
    }
    ep = sm.ep;
    eq = sm.eq;
    fp = sm.fp;
    fq = sm.fq;
    shift = 0;
  } else {
    if (bits(sm.pp) == 0ull || bits(sm.qq) == 0ull) {
      // a zero column: never rotated; swapped iff ||g_p|| < ||g_q||
      o.rot = false;
      o.swap = bits(sm.pp) < bits(sm.qq);
      return o;
    }
    // (e,f) norms: ||g_j|| = 2^e_j f_j, 1 <= f_j < 2
    const double rp = soft::sqrt_rn(sm.pp), rq = soft::sqrt_rn(sm.qq);
    ep = flg(rp);
    eq = flg(rq);
    fp = ldexp_rn(rp, -ep);
    fq = ldexp_rn(rq, -eq);
    shift = -(ep + eq);
  }
  // a21' = (g_q/2^eq)^* (g_p/2^ep) / (f_q f_p)
  const double d = __dmul_rn(fq, fp);
  const double zr = soft::div_rn(ldexp_rn(sm.qr, shift), d);
  const double zi = CPLX ? soft::div_rn(ldexp_rn(sm.qi, shift), d) : 0.0;
  const double az = CPLX ? hypot_naive(zr, zi) : dabs(zr);
  o.rot = !(ord(az) < ord(ups));
  // Alg. Gram
  const double q12 = soft::div_rn(fp, fq), q21 = soft::div_rn(fq, fp);
  double f12 = q12, f21 = q21;
  int e12 = ep - eq + flg(f12), e21 = eq - ep + flg(f21);
  f12 = ldexp_rn(f12, -flg(f12));
  f21 = ldexp_rn(f21, -flg(f21));
  const int sA = min(1023 - max(e12, e21), 0);
  const double b11 = ldexp_rn(f12, e12 + sA), b22 = ldexp_rn(f21, e21 + sA);
  const double b21r = ldexp_rn(zr, sA);
  Rot2 r;
  if (CPLX) {
    r = zsjac2<kMaskAllSoft>(b11, b22, b21r, ldexp_rn(zi, sA));
  } else {
    r = dsjac2<kMaskAllSoft>(b11, b22, b21r);
  }
  o.swap = perm_bit(r) != 0;
  o.c = r.cphi;
  o.C = r.etr;
  o.S = r.eti;
  gs_select(o, ep, eq, q12, q21, zr, zi, ups);
  return o;
}


// pair_rotation computed by a whole warp whose every lane holds the pair's
// sums: the same operations on the same operands, so the same bits, but the
// divisions and square roots that do not depend on one another run side by
// side, lane r (mod 4) taking the r-th of a stage as one warp instruction:
//   1 sqrt  ||g_p||^2, ||g_q||^2
//   2 div   Re a21', Im a21', f_p/f_q, f_q/f_p (Alg. zdpscl, Alg. Gram)
//   3 div   am/aM of Eq. e:zpolar; m/M of Alg. hypot for |a21'|      (complex)
//   4 sqrt  their sqrt(x^2 + 1)                                        (complex)
//   5 div   o/|a| of Eq. e:tan2; |Re a21'|/|a21'|, Im a21'/|a21'|
//   6 sqrt  sqrt(tan2^2 + 1)
//   7 div   tan(phi)
//   8 sqrt  sec(phi)
//   9 div   cos(phi); lambda1', lambda2'
// The chain of dependent correctly rounded operations is then 7 (real) or 9
// (complex) long instead of the 12 or 19 one lane would run.  For launches
// with one pair per warp, whose step time is this chain.  Since its lanes
// run different operations, the chain uses the select-based division,
// square root and x 2^k of fp64sel.cuh (same results, no divergent
// branches): real 7960 -> 6680 cycles per rotation, complex 10630 -> 9230.
// A lane whose stage has a zero divisor (a result the selects below then
// discard) divides by 1 instead.
template <bool CPLX>
__device__ __forceinline__ PairOut pair_rotation_warp(const PairSums &sm, double ups)
{
  const int r = threadIdx.x & 3;
  auto from = [](double x, int src) { return __shfl_sync(0xffffffffu, x, src); };
  PairOut o;
  o.c = 1.0;
  o.C = 0.0;
  o.S = 0.0;
  o.gs = 0;
  o.ex = o.ey = 0;
  o.psr = o.psi = o.psq = 0.0;
  int ep, eq, shift;
  double fp, fq;
  if (sm.wide) {
    if (sm.ep == kNegInfE || sm.eq == kNegInfE) {
      o.rot = false;
      o.swap = (sm.ep == kNegInfE) && (sm.eq != kNegInfE);
      return o;
    }
    ep = sm.ep;
    eq = sm.eq;
    fp = sm.fp;
    fq = sm.fq;
    shift = 0;
  } else {
    if (bits(sm.pp) == 0ull || bits(sm.qq) == 0ull) {
      o.rot = false;
      o.swap = bits(sm.pp) < bits(sm.qq);
      return o;
    }
    const double s1 = soft::sqrt_rn_sel(r == 0 ? sm.pp : sm.qq);  // stage 1
    const double rp = from(s1, 0), rq = from(s1, 1);
    // the square roots of positive normal sums are positive and normal:
    // their exponents and mantissas in [1, 2) straight from the bits
    ep = (int)(bits(rp) >> 52) - 1023;
    eq = (int)(bits(rq) >> 52) - 1023;
    fp = dbl((bits(rp) & kMant) | (1023ull << 52));
    fq = dbl((bits(rq) & kMant) | (1023ull << 52));
    shift = -(ep + eq);
  }
  // stage 2: a21' = (g_q/2^eq)^* (g_p/2^ep) / (f_q f_p), f_p/f_q, f_q/f_p
  const double d = __dmul_rn(fq, fp);
  const double sqr = soft::ldexp_rn_uni(sm.qr, shift);
  const double sqi = CPLX ? soft::ldexp_rn_uni(sm.qi, shift) : 1.0;
  const double n2 = (r == 0) ? sqr
                    : (r == 1) ? sqi
                    : (r == 2) ? fp : fq;
  const double d2 = (r == 0) ? d : (r == 1) ? (CPLX ? d : 1.0) : (r == 2) ? fq : fp;
  const double v2 = soft::div_rn_sel(n2, d2);
  const double zr = from(v2, 0), zi = CPLX ? from(v2, 1) : 0.0;
  const double q12 = from(v2, 2), q21 = from(v2, 3);
  // Alg. Gram, then Eq. e:z's scaling of the EVD (Alg. d8jac2 / Listing 1)
  double a11, a22, a21r, a21i;
  {
    // Every x 2^k here is exact while its result stays normal, which holds
    // for all but pairs whose norms are some 2^1000 apart: the scaling is
    // then done on the bit patterns (one check for the whole chain), and
    // otherwise by the same steps through ldexp_rn_uni.
    const uint64_t b12 = bits(q12), b21 = bits(q21);
    const int E12 = (int)(b12 >> 52), E21 = (int)(b21 >> 52);  // q12, q21 > 0
    const int e12 = ep - eq + E12 - 1023, e21 = eq - ep + E21 - 1023;  // exact if normal
    const int sA = min(1023 - max(e12, e21), 0);
    const unsigned long long x11 = ((unsigned long long)(1023 + e12) << 52) | (b12 & kMant);  // f12 2^e12
    const unsigned long long x22 = ((unsigned long long)(1023 + e21) << 52) | (b21 & kMant);
    const int zeta = 1020 - flg_sat(dbl(max(max(x11, x22), max(abits(zr), abits(zi)))));
    const unsigned long long zrb = abits(zr), zib = abits(zi);
    const int Er = (int)(zrb >> 52), Ei = (int)(zib >> 52);
    const bool fast = (unsigned)(E12 - 1) < 2046u && (unsigned)(E21 - 1) < 2046u && sA == 0 &&
                      e12 >= -1022 && e21 >= -1022 && (unsigned)(e12 + zeta + 1022) < 2046u &&
                      (unsigned)(e21 + zeta + 1022) < 2046u &&
                      (zrb == 0ull || ((unsigned)(Er - 1) < 2046u && (unsigned)(Er + zeta - 1) < 2046u)) &&
                      (zib == 0ull || ((unsigned)(Ei - 1) < 2046u && (unsigned)(Ei + zeta - 1) < 2046u));
    if (fast) {
      const unsigned long long kz = (unsigned long long)(long long)zeta << 52;
      a11 = dbl(x11 + kz);
      a22 = dbl(x22 + kz);
      a21r = zrb ? dbl(bits(zr) + kz) : zr;
      a21i = zib ? dbl(bits(zi) + kz) : zi;
    } else {
      const int g12 = flg(q12), g21 = flg(q21);
      const int h12 = ep - eq + g12, h21 = eq - ep + g21;
      const double f12 = soft::ldexp_rn_uni(q12, -g12), f21 = soft::ldexp_rn_uni(q21, -g21);
      const int tA = min(1023 - max(h12, h21), 0);
      a11 = soft::ldexp_rn_uni(f12, h12 + tA);
      a22 = soft::ldexp_rn_uni(f21, h21 + tA);
      a21r = soft::ldexp_rn_uni(zr, tA);
      a21i = CPLX ? soft::ldexp_rn_uni(zi, tA) : 0.0;
      const int z2 = 1020 - flg_max(a11, a22, a21r, a21i);  // a21i = 0 when real
      a11 = soft::ldexp_rn_uni(a11, z2);
      a22 = soft::ldexp_rn_uni(a22, z2);
      a21r = soft::ldexp_rn_uni(a21r, z2);
      if (CPLX) a21i = soft::ldexp_rn_uni(a21i, z2);
    }
  }
  double az, aa21, ar = dabs(a21r);
  bool zero = false;
  if (CPLX) {
    // stages 3, 4: |a21'| by Eq. e:zpolar (lane 0) and the convergence
    // test's hypot of the unscaled a21' (lane 1), side by side
    const double ai = dabs(a21i);
    const bool rmin = bits(ar) <= bits(ai);
    const double am = rmin ? ar : ai, aM = rmin ? ai : ar;
    zero = (bits(aM) == 0ull);
    const double azr = dabs(zr), azi = dabs(zi);
    const bool xm = bits(azr) <= bits(azi);
    const double mz = xm ? azr : azi, Mz = xm ? azi : azr;
    const bool zz = (bits(Mz) == 0ull);
    const double v3 = soft::div_rn_sel(r == 0 ? am : mz, r == 0 ? (zero ? 1.0 : aM) : (zz ? 1.0 : Mz));
    const double mM = zero ? 0.0 : from(v3, 0), qz = zz ? 0.0 : from(v3, 1);
    const double v4 = soft::sqrt_rn_sel(r == 0 ? __fma_rn(mM, mM, 1.0) : __fma_rn(qz, qz, 1.0));
    aa21 = __dmul_rn(from(v4, 0), aM);
    az = __dmul_rn(from(v4, 1), Mz);
  } else {
    aa21 = ar;
    az = dabs(zr);
  }
  o.rot = !(ord(az) < ord(ups));
  // stage 5: Eq. e:tan2's o/|a| (|a| = 0 gives Inf or NaN, which the clamp
  // turns into fl(sqrt nu) or 0), and the phase of a21'
  const double oo = twice_abs(aa21);
  const double a = __dsub_rn(a11, a22);
  const double aa = dabs(a);
  const double den21 = zero ? 1.0 : aa21;
  const double n5 = (r == 0) ? oo : (r == 1) ? ar : a21i;
  const double d5 = (r == 0) ? ((bits(aa) == 0ull) ? 1.0 : aa) : den21;
  const double v5 = soft::div_rn_sel(n5, CPLX ? d5 : ((bits(aa) == 0ull) ? 1.0 : aa));
  const double q5 = from(v5, 0);
  const double q = (bits(aa) == 0ull) ? ((bits(oo) == 0ull) ? 0.0 : dbl(kInf)) : q5;
  const double tan2 = clamp_tan2(q, a);
  // stages 6 - 8: tan(phi), sec^2(phi), sec(phi) (Eq. e:jactan, e:jacsec)
  const double tan1 = soft::div_rn_sel(tan2, __dadd_rn(1.0, soft::sqrt_rn_sel(__fma_rn(tan2, tan2, 1.0))));
  const double sec2 = __fma_rn(tan1, tan1, 1.0);
  const double sec = soft::sqrt_rn_sel(sec2);
  // stage 9: cos(phi) = 1/sec(phi); the eigenvalues of Eq. e:lamsec
  const double nl1 = __fma_rn(tan1, __fma_rn(a22, tan1, oo), a11);
  const double nl2 = __fma_rn(tan1, __fma_rn(a11, tan1, -oo), a22);
  const double v9 = soft::div_rn_sel((r == 0) ? 1.0 : (r == 1) ? nl1 : nl2, (r == 0) ? sec : sec2);
  const double cphi = from(v9, 0), l1s = from(v9, 1), l2s = from(v9, 2);
  if (CPLX) {
    const double qc = from(v5, 1), qs = from(v5, 2);
    const double ca = with_sign(zero ? 1.0 : qc, a21r);  // fmin(., 1)
    const double sa = zero ? a21i : qs;
    o.C = __dmul_rn(ca, tan1);
    o.S = __dmul_rn(sa, tan1);
  } else {
    o.C = xor_sign(tan1, a21r);
    o.S = 0.0;
  }
  o.c = cphi;
  o.swap = ord(l1s) < ord(l2s);
  gs_select(o, ep, eq, q12, q21, zr, zi, ups);
  return o;
}

// The compensated dot-product of supplement SM2.2 (Alg. zdpscl' /
// ddpscl'): each term x y enters as c = RD(x y) and c' = x y - c >= 0 (one
// fma, exact), and each of the two streams is summed by Kahan's method
// with 2Sum (Eq. e:d2sum) in place of Fast2Sum.
struct CompSum {
  double s, t;    // value stream and its carried error
  double s2, t2;  // error stream and its carried error
};

// Eq. e:d2sum: a + b = s + t exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &t)
{
  const double ss = __dadd_rn(a, b);
  double a1 = __dsub_rn(ss, b);
  double b1 = __dsub_rn(ss, a1);
  a1 = __dsub_rn(a, a1);
  b1 = __dsub_rn(b, b1);
  s = ss;
  t = __dadd_rn(a1, b1);
}

__device__ __forceinline__ void comp_term(double x, double y, CompSum &c)
{
  const double p = __dmul_rd(x, y);
  const double e = __fma_rn(x, y, -p);
  two_sum(c.s, __dadd_rn(p, c.t), c.s, c.t);
  two_sum(c.s2, __dadd_rn(e, c.t2), c.s2, c.t2);
}

// The lanes' streams reduced one by one in the canonical butterfly order,
// then combined as s + (t + (s' + t')).
__device__ __forceinline__ double comp_reduce(const CompSum &c)
{
  const double S = warp_sum(c.s), T = warp_sum(c.t), S2 = warp_sum(c.s2), T2 = warp_sum(c.t2);
  return __dadd_rn(S, __dadd_rn(T, __dadd_rn(S2, T2)));
}

// Bit pattern of 2^-969: a sum of squares below it may contain squares
// that fell below the normal range (2^-1022) with more than a negligible
// part of their bits lost.
constexpr unsigned long long kWideBelow = 0x0360000000000000ull;

// The pair's sums for columns with tiny entries (supplement SM6 and
// Alg. zdpscl as printed): pass 1 takes the columns' norms with the
// wide-exponent method of Alg. rnF, pass 2 the dot-product of the columns
// prescaled by 2^-e_j (in the canonical lane order, compensated if COMP).
// FP64 columns only.
template <bool CPLX, int CG, bool COMP>
__device__ __noinline__ PairSums pair_sums_wide(const MatViewT<double, CG> &M, int p, int q)
{
  const int lane = threadIdx.x & 31;
  const double *gpr = M.Gr(p), *gqr = M.Gr(q);
  const double *gpi = CPLX ? M.Gi(p) : nullptr, *gqi = CPLX ? M.Gi(q) : nullptr;
  EF np = {kNegInfE, 1.0}, nq = {kNegInfE, 1.0};
  for (int i = lane; i < M.mp; i += 32) {
    ef_fma_step(M.ld(gpr + i), np);
    ef_fma_step(M.ld(gqr + i), nq);
    if (CPLX) {
      ef_fma_step(M.ld(gpi + i), np);
      ef_fma_step(M.ld(gqi + i), nq);
    }
  }
  np = ef_sqrt(ef_warp_sum(np));
  nq = ef_sqrt(ef_warp_sum(nq));
  PairSums r;
  r.pp = r.qq = 0.0;
  r.qr = r.qi = 0.0;
  r.ep = np.e;
  r.fp = np.f;
  r.eq = nq.e;
  r.fq = nq.f;
  r.wide = 1;
  if (np.e == kNegInfE || nq.e == kNegInfE) return r;
  double sqr = 0.0, sqi = 0.0;
  CompSum cr = {0.0, 0.0, 0.0, 0.0}, ci = {0.0, 0.0, 0.0, 0.0};
  for (int i = lane; i < M.mp; i += 32) {
    const double xpr = ldexp_rn(M.ld(gpr + i), -np.e), xqr = ldexp_rn(M.ld(gqr + i), -nq.e);
    const double xpi = CPLX ? ldexp_rn(M.ld(gpi + i), -np.e) : 0.0;
    const double xqi = CPLX ? ldexp_rn(M.ld(gqi + i), -nq.e) : 0.0;
    if constexpr (COMP) {
      comp_term(xpr, xqr, cr);
      if (CPLX) {
        comp_term(xpi, xqi, cr);
        comp_term(xpi, xqr, ci);
        comp_term(-xpr, xqi, ci);
      }
    } else {
      sqr = __fma_rn(xqr, xpr, sqr);
      if (CPLX) {
        sqi = __fma_rn(xqr, xpi, sqi);
        sqr = __fma_rn(xqi, xpi, sqr);
        sqi = __fma_rn(-xqi, xpr, sqi);
      }
    }
  }
  if constexpr (COMP) {
    r.qr = comp_reduce(cr);
    r.qi = CPLX ? comp_reduce(ci) : 0.0;
  } else {
    r.qr = warp_sum(sqr);
    r.qi = CPLX ? warp_sum(sqi) : 0.0;
  }
  return r;
}

// The three sums of pair (p, q), formed by one full warp with the columns
// in precision T (double, or float in the FP32 phase of the mixed SVD):
// lane l accumulates rows l, l+32, ... in ascending order with fma, the lane
// partials are combined in FP64 by warp_sum_slots (the same values end up
// in every lane).  rk != 0 downscales both columns of G by 2^rk first (section 3.2,
// step 2; FP64 only).  COMP forms g_q^* g_p by the compensated summation
// (FP64 only); the squared norms stay plain fma sums.
template <typename T, bool CPLX, int CG, bool COMP = false, int U = (sizeof(T) == 4) ? 8 : 4>
__device__ __forceinline__ PairSums pair_sums(const MatViewT<T, CG> &M, int p, int q, int rk)
{
  static_assert(!COMP || sizeof(T) == 8, "the compensated sums are FP64 only");
  // U rows per lane per loop trip: their loads are all issued before the
  // arithmetic, which then consumes them in ascending row order, so the
  // accumulation order (and the bits) are those of the one-row loop.  The
  // rows of a last, partial trip cost FP64 issue slots all the same (a
  // masked FP64 instruction takes the pipe like a full one): wide trips
  // only where the column fills them.
  const int lane = threadIdx.x & 31;
  T *gpr = M.Gr(p), *gqr = M.Gr(q);
  T *gpi = CPLX ? M.Gi(p) : nullptr, *gqi = CPLX ? M.Gi(q) : nullptr;
  T spp = T(0), sqq = T(0), sqr = T(0), sqi = T(0);
  CompSum cr = {0.0, 0.0, 0.0, 0.0}, ci = {0.0, 0.0, 0.0, 0.0};
  for (int base = lane; base < M.mp; base += 32 * U) {
    T xpr[U], xqr[U], xpi[U], xqi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + 32 * u;  // the same bound for every lane: mp is a multiple of 32
      xpr[u] = xqr[u] = xpi[u] = xqi[u] = T(0);
      if (i < M.mp) {
        xpr[u] = M.ld(gpr + i);
        xqr[u] = M.ld(gqr + i);
        if (CPLX) {
          xpi[u] = M.ld(gpi + i);
          xqi[u] = M.ld(gqi + i);
        }
      }
    }
    if (rk) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = base + 32 * u;
        if (i < M.mp) {
          xpr[u] = ldexp_rn(xpr[u], rk);
          xqr[u] = ldexp_rn(xqr[u], rk);
          M.st(gpr + i, xpr[u]);
          M.st(gqr + i, xqr[u]);
          if (CPLX) {
            xpi[u] = ldexp_rn(xpi[u], rk);
            xqi[u] = ldexp_rn(xqi[u], rk);
            M.st(gpi + i, xpi[u]);
            M.st(gqi + i, xqi[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (base + 32 * u < M.mp) {
        spp = fma_t(xpr[u], xpr[u], spp);
        sqq = fma_t(xqr[u], xqr[u], sqq);
        if constexpr (COMP) {
          // Re: g_p.re g_q.re + g_p.im g_q.im; Im: g_p.im g_q.re - g_p.re g_q.im
          comp_term(xpr[u], xqr[u], cr);
          if (CPLX) {
            spp = fma_t(xpi[u], xpi[u], spp);
            sqq = fma_t(xqi[u], xqi[u], sqq);
            comp_term(xpi[u], xqi[u], cr);
            comp_term(xpi[u], xqr[u], ci);
            comp_term(-xpr[u], xqi[u], ci);
          }
        } else {
          sqr = fma_t(xqr[u], xpr[u], sqr);
          if (CPLX) {
            spp = fma_t(xpi[u], xpi[u], spp);
            sqq = fma_t(xqi[u], xqi[u], sqq);
            sqi = fma_t(xqr[u], xpi[u], sqi);
            sqr = fma_t(xqi[u], xpi[u], sqr);
            sqi = fma_t(-xqi[u], xpr[u], sqi);
          }
        }
      }
    }
  }
  // the lane partials combined in FP64 by one tree for all the sums
  PairSums r;
  if constexpr (COMP) {
    double v[16] = {(double)spp, (double)sqq, cr.s, cr.t, cr.s2, cr.t2, ci.s, ci.t,
                    ci.s2, ci.t2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double x = warp_sum_slots<16>(v);
    r.pp = warp_slot<16>(x, 0);
    r.qq = warp_slot<16>(x, 1);
    // s + (t + (s' + t')) per component
    r.qr = __dadd_rn(warp_slot<16>(x, 2),
                     __dadd_rn(warp_slot<16>(x, 3),
                               __dadd_rn(warp_slot<16>(x, 4), warp_slot<16>(x, 5))));
    r.qi = CPLX ? __dadd_rn(warp_slot<16>(x, 6),
                            __dadd_rn(warp_slot<16>(x, 7),
                                      __dadd_rn(warp_slot<16>(x, 8), warp_slot<16>(x, 9))))
                : 0.0;
  } else {
    double v[4] = {(double)spp, (double)sqq, (double)sqr, (double)sqi};
    const double x = warp_sum_slots<4>(v);
    r.pp = warp_slot<4>(x, 0);
    r.qq = warp_slot<4>(x, 1);
    r.qr = warp_slot<4>(x, 2);
    r.qi = CPLX ? warp_slot<4>(x, 3) : 0.0;
  }
  r.fp = r.fq = 1.0;
  r.ep = r.eq = 0;
  r.wide = 0;
  if constexpr (sizeof(T) == 8) {
    // squares below 2^-1022 may have lost bits: a column whose squared norm
    // is below 2^-969 is redone with the wide-exponent norms (the same
    // decision in every lane)
    if (bits(r.pp) < kWideBelow || bits(r.qq) < kWideBelow)
      r = pair_sums_wide<CPLX, CG, COMP>(M, p, q);
  }
  return r;
}

// Eq. e:GS (Alg. ZGS / DGS, in their operation order) on G: the target
// column y <- (y / 2^ey - psi x / 2^ex) 2^ey, the source x unchanged, the
// pair swapped afterwards if o.swap; Mloc takes the max-norm of both new
// columns.  One full warp, FP64 columns.
template <bool CPLX, int CG>
__device__ __forceinline__ void gs_apply(const MatViewT<double, CG> &M, int p, int q,
                                         const PairOut &o, unsigned long long &Mloc)
{
  const int lane = threadIdx.x & 31;
  const int src = (o.gs == 1) ? p : q, dst = (o.gs == 1) ? q : p;
  double *xr = M.Gr(src), *yr = M.Gr(dst);
  double *xi = CPLX ? M.Gi(src) : nullptr, *yi = CPLX ? M.Gi(dst) : nullptr;
  // with the swap the new target lands in the source's place and back
  double *ox_r = o.swap ? yr : xr, *oy_r = o.swap ? xr : yr;
  double *ox_i = o.swap ? yi : xi, *oy_i = o.swap ? xi : yi;
  const double psr = __dmul_rn(o.psr, o.psq), psi = __dmul_rn(o.psi, o.psq);
  for (int i = lane; i < M.mp; i += 32) {
    const double x1 = M.ld(xr + i), y1 = M.ld(yr + i);
    const double sx1 = ldexp_rn(x1, -o.ex), sy1 = ldexp_rn(y1, -o.ey);
    if (CPLX) {
      const double x2 = M.ld(xi + i), y2 = M.ld(yi + i);
      const double sx2 = ldexp_rn(x2, -o.ex), sy2 = ldexp_rn(y2, -o.ey);
      const double nr = ldexp_rn(__fma_rn(-psr, sx1, __fma_rn(psi, sx2, sy1)), o.ey);
      const double ni = ldexp_rn(__fma_rn(-psr, sx2, __fma_rn(-psi, sx1, sy2)), o.ey);
      M.st(ox_r + i, x1);
      M.st(ox_i + i, x2);
      M.st(oy_r + i, nr);
      M.st(oy_i + i, ni);
      Mloc = max(Mloc, max(max(magbits(x1), magbits(x2)), max(magbits(nr), magbits(ni))));
    } else {
      const double nr = ldexp_rn(__fma_rn(-psr, sx1, sy1), o.ey);
      M.st(ox_r + i, x1);
      M.st(oy_r + i, nr);
      Mloc = max(Mloc, max(magbits(x1), magbits(nr)));
    }
  }
}

// One row of Eq. e:transf: x_p' = fma(x_q, e', x_p) c, x_q' = fma(x_p,
// -conj(e'), x_q) c, e' = C + iS (real: S = 0).
template <typename T, bool CPLX>
__device__ __forceinline__ void rotate_row(T pr, T pi, T qr, T qi, T c, T C, T S, T &npr, T &npi,
                                           T &nqr, T &nqi)
{
  if (CPLX) {
    npr = mul_t(fma_t(qr, C, fma_t(-qi, S, pr)), c);
    npi = mul_t(fma_t(qr, S, fma_t(qi, C, pi)), c);
    nqr = mul_t(fma_t(pr, -C, fma_t(-pi, S, qr)), c);
    nqi = mul_t(fma_t(pr, S, fma_t(pi, -C, qi)), c);
  } else {
    npr = mul_t(fma_t(qr, C, pr), c);
    nqr = mul_t(fma_t(pr, -C, qr), c);
    npi = nqi = T(0);
  }
}

// Eq. e:transf (Alg. zjrot) on the pair's G rows (tracking the max-norm of
// the new entries in Mloc, as magbits() in T's encoding) and V rows, with the
// columns swapped if o.swap; a non-rotated pair with o.swap is only swapped.
// One full warp; o must be the same in every lane.  U rows per lane per
// loop trip, whose loads are all issued before its arithmetic and stores
// (the rows are independent, so U changes no bits).  G's rows and then V's
// take separate trips; with MERGED, G's mp rows followed by V's np rows are
// one sequence (both multiples of 32, so each 32 rows lie in one matrix),
// so that a trip may hold rows of both -- one trip for a short pair of
// columns, at the price of a pointer select per row.  G_ONLY leaves V to the
// caller (DeferredV).
template <typename T, bool CPLX, int CG, int U = (sizeof(T) == 4) ? 8 : 4, bool MERGED = false,
          bool G_ONLY = false>
__device__ __forceinline__ void pair_apply(const MatViewT<T, CG> &M, int p, int q, const PairOut &o,
                                           unsigned long long &Mloc)
{
  const int lane = threadIdx.x & 31;
  const bool swp = o.swap;
  if (o.rot) {
    const T c = to_t(o.c, T(0)), C = to_t(o.C, T(0));
    const T S = CPLX ? to_t(o.S, T(0)) : T(0);
    bool gdone = false;
    if constexpr (sizeof(T) == 8) {
      if (o.gs) {  // Eq. e:GS replaces the rotation on G
        gs_apply<CPLX, CG>(M, p, q, o, Mloc);
        gdone = true;
      }
    }
    // x_p' = fma(x_q, e', x_p) c, x_q' = fma(x_p, -conj(e'), x_q) c, e' = C + iS
    auto rotate = [&](const T pr, const T pi, const T qr, const T qi, T *dpr, T *dpi, T *dqr,
                      T *dqi, bool onG) {
      T npr, npi, nqr, nqi;
      rotate_row<T, CPLX>(pr, pi, qr, qi, c, C, S, npr, npi, nqr, nqi);
      M.st(dpr, npr);
      M.st(dqr, nqr);
      if (CPLX) {
        M.st(dpi, npi);
        M.st(dqi, nqi);
        if (onG) {
          const unsigned long long a =
              max(max(magbits(npr), magbits(npi)), max(magbits(nqr), magbits(nqi)));
          Mloc = max(Mloc, a);
        }
      } else {
        if (onG) Mloc = max(Mloc, max(magbits(npr), magbits(nqr)));
      }
    };
    T *gpr = M.Gr(p), *gqr = M.Gr(q);
    T *vpr = M.Vr(p), *vqr = M.Vr(q);
    T *gpi = CPLX ? M.Gi(p) : nullptr, *gqi = CPLX ? M.Gi(q) : nullptr;
    T *vpi = CPLX ? M.Vi(p) : nullptr, *vqi = CPLX ? M.Vi(q) : nullptr;
    if constexpr (MERGED) {
      // G's trips from the last to the first (the sums just read those rows
      // in ascending order, so the latest are the likeliest still in L2),
      // then V's in order; the rows are independent, so the order changes
      // no bits
      const int r0 = gdone ? M.mp : 0, R = G_ONLY ? M.mp : M.mp + M.np;
      const int ntrip = (R - r0 + 32 * U - 1) / (32 * U);
      const int ntg = (M.mp - r0 + 32 * U - 1) / (32 * U);  // trips that start in G
      for (int j = 0; j < ntrip; ++j) {
        const int base = r0 + lane + 32 * U * ((j < ntg) ? ntg - 1 - j : j);
        T pr[U], qr[U], pi[U], qi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int v = base + 32 * u;
          pr[u] = qr[u] = pi[u] = qi[u] = T(0);
          if (v < R) {
            const bool onG = v < M.mp;
            const int i = onG ? v : v - M.mp;
            pr[u] = M.ld((onG ? gpr : vpr) + i);
            qr[u] = M.ld((onG ? gqr : vqr) + i);
            if (CPLX) {
              pi[u] = M.ld((onG ? gpi : vpi) + i);
              qi[u] = M.ld((onG ? gqi : vqi) + i);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int v = base + 32 * u;
          if (v < R) {
            const bool onG = v < M.mp;
            const int i = onG ? v : v - M.mp;
            T *xpr = onG ? gpr : vpr, *xqr = onG ? gqr : vqr;
            T *xpi = onG ? gpi : vpi, *xqi = onG ? gqi : vqi;
            T *dpr = (swp ? xqr : xpr) + i, *dqr = (swp ? xpr : xqr) + i;
            T *dpi = CPLX ? (swp ? xqi : xpi) + i : nullptr, *dqi = CPLX ? (swp ? xpi : xqi) + i : nullptr;
            rotate(pr[u], pi[u], qr[u], qi[u], dpr, dpi, dqr, dqi, onG);
          }
        }
      }
    } else {
      for (int pass = gdone ? 1 : 0; pass < (G_ONLY ? 1 : 2); ++pass) {
        const bool onG = (pass == 0);
        const int rows = onG ? M.mp : M.np;
        T *xpr = onG ? gpr : vpr, *xqr = onG ? gqr : vqr;
        T *xpi = onG ? gpi : vpi, *xqi = onG ? gqi : vqi;
        T *dpr = swp ? xqr : xpr, *dqr = swp ? xpr : xqr;
        T *dpi = swp ? xqi : xpi, *dqi = swp ? xpi : xqi;
        for (int base = lane; base < rows; base += 32 * U) {
          T pr[U], qr[U], pi[U], qi[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = base + 32 * u;
            pr[u] = qr[u] = pi[u] = qi[u] = T(0);
            if (i < rows) {
              pr[u] = M.ld(xpr + i);
              qr[u] = M.ld(xqr + i);
              if (CPLX) {
                pi[u] = M.ld(xpi + i);
                qi[u] = M.ld(xqi + i);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = base + 32 * u;
            if (i < rows)
              rotate(pr[u], pi[u], qr[u], qi[u], dpr + i, CPLX ? dpi + i : nullptr, dqr + i,
                     CPLX ? dqi + i : nullptr, onG);
          }
        }
      }
    }
  } else if (swp) {
    for (int pass = 0; pass < (G_ONLY ? 1 : 2); ++pass) {
      const bool onG = (pass == 0);
      const int rows = onG ? M.mp : M.np;
      T *xpr = onG ? M.Gr(p) : M.Vr(p);
      T *xqr = onG ? M.Gr(q) : M.Vr(q);
      T *xpi = CPLX ? (onG ? M.Gi(p) : M.Vi(p)) : nullptr;
      T *xqi = CPLX ? (onG ? M.Gi(q) : M.Vi(q)) : nullptr;
      for (int i = lane; i < rows; i += 32) {
        const T a = M.ld(xpr + i), b = M.ld(xqr + i);
        M.st(xpr + i, b);
        M.st(xqr + i, a);
        if (CPLX) {
          const T ai = M.ld(xpi + i), bi = M.ld(xqi + i);
          M.st(xpi + i, bi);
          M.st(xqi + i, ai);
        }
      }
    }
  }
  __syncwarp();
}

// One chunk of CH <= 32 pivot pairs (l = base .. base + CH - 1) of step k,
// executed by the whole block (W warps, three block barriers):
//   1. warps form the sums of the chunk's pairs,
//   2. one thread per pair turns them into the rotation (Alg. zdpscl's
//      division, Alg. cvg, Alg. Gram, the EVD) -- the narrow FP64 pipe
//      charges a masked warp instruction like a full one, so the EVDs of
//      the chunk share their instructions instead of one lane each,
//   3. warps apply the rotations.
// Every pair's arithmetic is the same whatever the chunking.  rots counts
// (in each warp's lane 0) the transformed pairs and gsn those of them that
// took the Gram-Schmidt step; Mloc collects magbits().
template <typename T, bool CPLX, int CG, bool COMP = false>
__device__ __forceinline__ void step_chunk(const MatViewT<T, CG> &M, int k, int nt, int base, int CH,
                                           double ups, int rk, bool permute, PairSums *s_sums,
                                           PairOut *s_out, unsigned long long &Mloc, int &rots,
                                           int &gsn, int *lastmod = nullptr, int gstep = 0,
                                           int last_rescale = 0)
{
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int L = nt / 2, K = nt - 1;
  constexpr int kSkipped = 2;  // PairSums::wide of a pair skipped as unchanged (step_warps)
  for (int i = warp; i < CH; i += W) {
    const int l = base + i;
    if (l >= L) break;
    int p, q;
    pair_of(k, l, nt, p, q);
    bool skip = false;
    if (lastmod != nullptr && q < M.n && rk == 0 && gstep - K > last_rescale) {
      const int before = gstep - K;  // the pair's last meeting, one sweep ago
      skip = __ldcg(lastmod + p) < before && __ldcg(lastmod + q) < before;
    }
    if (skip) {
      if (lane == 0) s_sums[i].wide = kSkipped;
    } else if (q < M.n) {
      const PairSums sm = pair_sums<T, CPLX, CG, COMP>(M, p, q, rk);
      if (lane == 0) s_sums[i] = sm;
    } else if (rk) {  // phantom partner: only a pending rescale applies
      scale_col(M, M.Gr(p), rk, lane);
      if (CPLX) scale_col(M, M.Gi(p), rk, lane);
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < CH) {
    const int i = threadIdx.x, l = base + i;
    if (l < L) {
      int p, q;
      pair_of(k, l, nt, p, q);
      if (q < M.n) {
        const PairSums sm = s_sums[i];
        PairOut o;
        if (sm.wide == kSkipped) {  // unchanged since its last meeting: no rotation, no swap
          o.rot = o.swap = false;
          o.c = 1.0;
          o.C = o.S = 0.0;
          o.gs = o.ex = o.ey = 0;
          o.psr = o.psi = o.psq = 0.0;
        } else {
          o = pair_rotation<CPLX>(sm, ups);
          o.swap = o.swap && permute;
        }
        s_out[i] = o;
      }
    }
  }
  __syncthreads();
  for (int i = warp; i < CH; i += W) {
    const int l = base + i;
    if (l >= L) break;
    int p, q;
    pair_of(k, l, nt, p, q);
    if (q < M.n) {
      const PairOut o = s_out[i];
      pair_apply<T, CPLX>(M, p, q, o, Mloc);
      if (lane == 0 && o.rot) ++rots;
      if (lane == 0 && o.gs) ++gsn;
      if (lastmod != nullptr && lane == 0 && (o.rot || o.swap)) {
        __stcg(lastmod + p, gstep);
        __stcg(lastmod + q, gstep);
      }
    }
  }
  __syncthreads();
}

// A pair's transformation of V held over to the next step.  The sweep
// never reads V but to transform it, and V's columns p and q are not
// touched by any other pair before the next step's barrier, so applying
// step k's rotation to them during step k + 1 keeps every column's updates
// in their order and gives the same bits.  The rows (np <= 32 kRows per
// lane: one trip) are loaded before the next rotation's chain of dependent
// operations and transformed after it, so their L2 round trip is hidden
// behind that chain and the step's critical path keeps only G's rows.
template <typename T, bool CPLX>
struct DeferredV {
  static constexpr int kRows = 4;
  int p = -1, q = -1;  // the pending pair (p < 0: none)
  PairOut o;
  T pr[kRows], qr[kRows], pi[kRows], qi[kRows];

  template <int CG>
  __device__ __forceinline__ void load(const MatViewT<T, CG> &M)
  {
    const int lane = threadIdx.x & 31;
    const T *xp = M.Vr(p), *xq = M.Vr(q);
    const T *xpi = CPLX ? M.Vi(p) : nullptr, *xqi = CPLX ? M.Vi(q) : nullptr;
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int i = lane + 32 * u;
      pr[u] = qr[u] = pi[u] = qi[u] = T(0);
      if (i < M.np) {
        pr[u] = M.ld(xp + i);
        qr[u] = M.ld(xq + i);
        if (CPLX) {
          pi[u] = M.ld(xpi + i);
          qi[u] = M.ld(xqi + i);
        }
      }
    }
  }

  // the transformation (or the swap alone) of the loaded rows, as
  // pair_apply's V pass would do it
  template <int CG>
  __device__ __forceinline__ void apply(const MatViewT<T, CG> &M)
  {
    const int lane = threadIdx.x & 31;
    T *xp = M.Vr(p), *xq = M.Vr(q);
    T *xpi = CPLX ? M.Vi(p) : nullptr, *xqi = CPLX ? M.Vi(q) : nullptr;
    T *dp = o.swap ? xq : xp, *dq = o.swap ? xp : xq;
    T *dpi = o.swap ? xqi : xpi, *dqi = o.swap ? xpi : xqi;
    const T c = to_t(o.c, T(0)), C = to_t(o.C, T(0)), S = CPLX ? to_t(o.S, T(0)) : T(0);
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int i = lane + 32 * u;
      if (i < M.np) {
        T npr = pr[u], npi = pi[u], nqr = qr[u], nqi = qi[u];
        if (o.rot) rotate_row<T, CPLX>(pr[u], pi[u], qr[u], qi[u], c, C, S, npr, npi, nqr, nqi);
        M.st(dp + i, npr);
        M.st(dq + i, nqr);
        if (CPLX) {
          M.st(dpi + i, npi);
          M.st(dqi + i, nqi);
        }
      }
    }
    p = q = -1;
  }
};

// A block's share of step k when every warp runs its pairs alone: warp w
// takes pairs l = blockIdx.x W + w, + gridDim.x W, ..., each one its sums,
// its rotation (pair_rotation_warp, the same bits as the chunked form) and
// its transformation, with no block barrier in between.  For the
// persistent single-matrix sweep, where a step has at most a few pairs per
// block and its time is the chain of one pair.
//
// Unchanged pairs (lastmod != nullptr): lastmod[j] is the last global step
// (gstep counts the steps of the launch) at which column j was transformed,
// swapped or rescaled (-1: never).  A pair met again one sweep (K = nt - 1
// steps) after its last meeting with neither column changed since, and no
// rescaling since (last_rescale), has the same columns bit for bit, so its
// rotation test fails again: it is skipped, with the same results.
template <typename T, bool CPLX, bool COMP = false, int CG = kAccL2>
__device__ __forceinline__ void step_warps(const MatViewT<T, CG> &M, int k, int nt, double ups, int rk,
                                           bool permute, unsigned long long &Mloc, int &rots, int &gsn,
                                           bool defer, DeferredV<T, CPLX> &dv, int *lastmod = nullptr,
                                           int gstep = 0, int last_rescale = 0)
{
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int L = nt / 2;
  const int K = nt - 1;
  for (int l = blockIdx.x * W + warp; l < L; l += gridDim.x * W) {
    int p, q;
    pair_of(k, l, nt, p, q);
    bool skip = false;
    if (lastmod != nullptr && q < M.n && rk == 0 && gstep - K > last_rescale) {
      const int before = gstep - K;  // the pair's last meeting
      skip = __ldcg(lastmod + p) < before && __ldcg(lastmod + q) < before;
    }
    if (skip) {
      if (defer && dv.p >= 0) {  // settle the last step's V
        dv.load(M);
        dv.apply(M);
      }
    } else if (q < M.n) {
      // FP64 columns that fill them take wider load trips: sums 8 rows per
      // lane (4 complex), the transformation 12 (6 complex) of G's and V's
      // rows together -- one trip each for 256 + 128 rows
      constexpr int US = CPLX ? 4 : 8, UA = CPLX ? 6 : 12;
      const bool wide_sums = sizeof(T) == 8 && M.mp % (32 * US) == 0;
      const bool wide_apply = sizeof(T) == 8 && (M.mp + M.np) % (32 * UA) == 0;
      const PairSums sm = wide_sums ? pair_sums<T, CPLX, CG, COMP, US>(M, p, q, rk)
                                    : pair_sums<T, CPLX, CG, COMP>(M, p, q, rk);
      if (defer && dv.p >= 0) dv.load(M);  // the last step's V rows, in flight during the rotation
      PairOut o = pair_rotation_warp<CPLX>(sm, ups);
      o.swap = o.swap && permute;
      if (defer) {
        if (dv.p >= 0) dv.apply(M);
        if (wide_sums)
          pair_apply<T, CPLX, CG, US, false, true>(M, p, q, o, Mloc);
        else
          pair_apply<T, CPLX, CG, (sizeof(T) == 4) ? 8 : 4, false, true>(M, p, q, o, Mloc);
        if (o.rot || o.swap) {
          dv.p = p;
          dv.q = q;
          dv.o = o;
        }
      } else if (wide_apply) {
        pair_apply<T, CPLX, CG, UA, true>(M, p, q, o, Mloc);
      } else {
        pair_apply<T, CPLX, CG>(M, p, q, o, Mloc);
      }
      if (lane == 0 && o.rot) ++rots;
      if (lane == 0 && o.gs) ++gsn;
      if (lastmod != nullptr && lane == 0 && (o.rot || o.swap)) {
        __stcg(lastmod + p, gstep);
        __stcg(lastmod + q, gstep);
      }
    } else {
      if (defer && dv.p >= 0) {  // no pair of its own this step: settle the last one's V
        dv.load(M);
        dv.apply(M);
      }
      if (rk) {  // phantom partner: only a pending rescale applies
        scale_col(M, M.Gr(p), rk, lane);
        if (CPLX) scale_col(M, M.Gi(p), rk, lane);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// A step of a small matrix with four warps of a block on each pivot pair.
// A warp issues at most one FP64 instruction every few dozen cycles (on
// GB300 about 64), whatever their dependences, so a step whose time is one
// pair's chain is shortened by spreading the pair's FP64 instructions over
// four warps, which sit on the SM's four schedulers:
//   - every warp loads the pair's G rows (lane l: rows l, l + 32, ...) and
//     forms ONE of the sums (warp 0 ||g_p||^2, 1 ||g_q||^2, 2 Re g_q^* g_p,
//     3 Im g_q^* g_p) over them in the canonical order, reduced by the
//     butterfly warp_sum -- bit for bit the slot of pair_sums' tree;
//   - every warp computes the same rotation (pair_rotation_warp);
//   - warp g transforms the G rows u = g, g + 4, ... of its lanes from the
//     registers it loaded, and V's rows likewise one step late (GroupV).
// The columns' values, the sums and the rotations are those of the other
// step forms, so are the bits.  FP64 columns, plain sums; mp <= 32 U rows.
constexpr int kGroupWarps = 4;

template <bool CPLX>
struct GroupV {
  static constexpr int kRows = 2;  // V rows per lane and warp: np <= 32 * 4 * kRows
  int p = -1, q = -1;
  PairOut o;
  double pr[kRows], qr[kRows], pi[kRows], qi[kRows];

  template <int CG>
  __device__ __forceinline__ void load(const MatViewT<double, CG> &M, int g)
  {
    const int lane = threadIdx.x & 31;
    const double *xp = M.Vr(p), *xq = M.Vr(q);
    const double *xpi = CPLX ? M.Vi(p) : nullptr, *xqi = CPLX ? M.Vi(q) : nullptr;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = lane + 32 * (g + kGroupWarps * r);
      pr[r] = qr[r] = pi[r] = qi[r] = 0.0;
      if (i < M.np) {
        pr[r] = M.ld(xp + i);
        qr[r] = M.ld(xq + i);
        if (CPLX) {
          pi[r] = M.ld(xpi + i);
          qi[r] = M.ld(xqi + i);
        }
      }
    }
  }

  template <int CG>
  __device__ __forceinline__ void apply(const MatViewT<double, CG> &M, int g)
  {
    const int lane = threadIdx.x & 31;
    double *xp = M.Vr(p), *xq = M.Vr(q);
    double *xpi = CPLX ? M.Vi(p) : nullptr, *xqi = CPLX ? M.Vi(q) : nullptr;
    double *dp = o.swap ? xq : xp, *dq = o.swap ? xp : xq;
    double *dpi = o.swap ? xqi : xpi, *dqi = o.swap ? xpi : xqi;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = lane + 32 * (g + kGroupWarps * r);
      if (i < M.np) {
        double npr, npi, nqr, nqi;  // a swap without rotation stores the rows as they are
        rotate_row<double, CPLX>(pr[r], pi[r], qr[r], qi[r], o.c, o.C, o.S, npr, npi, nqr, nqi);
        M.st(dp + i, o.rot ? npr : pr[r]);
        M.st(dq + i, o.rot ? nqr : qr[r]);
        if (CPLX) {
          M.st(dpi + i, o.rot ? npi : pi[r]);
          M.st(dqi + i, o.rot ? nqi : qi[r]);
        }
      }
    }
    p = q = -1;
  }
};

// The block's pairs of step k (l = blockIdx.x, + gridDim.x, ...), each by
// the block's four warps; s_sum: four doubles of shared memory.
template <bool CPLX, int CG>
__device__ __forceinline__ void step_group(const MatViewT<double, CG> &M, int k, int nt, double ups,
                                           int rk, bool permute, unsigned long long &Mloc, int &rots,
                                           int &gsn, GroupV<CPLX> &gv, double *s_sum)
{
  constexpr int U = CPLX ? 4 : 8;  // G rows per lane: mp <= 32 U
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int L = nt / 2;
  const int urows = M.mp >> 5;  // rows per lane (mp is a multiple of 32)
  for (int l = blockIdx.x; l < L; l += gridDim.x) {
    int p, q;
    pair_of(k, l, nt, p, q);
    if (q >= M.n) {
      if (gv.p >= 0) {  // no pair this step: settle the last one's V
        gv.load(M, g);
        gv.apply(M, g);
      }
      if (rk && g == 0) {  // phantom partner: only a pending rescale applies
        scale_col(M, M.Gr(p), rk, lane);
        if (CPLX) scale_col(M, M.Gi(p), rk, lane);
      }
      continue;
    }
    double *gpr = M.Gr(p), *gqr = M.Gr(q);
    double *gpi = CPLX ? M.Gi(p) : nullptr, *gqi = CPLX ? M.Gi(q) : nullptr;
    double xpr[U], xqr[U], xpi[U], xqi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = lane + 32 * u;
      xpr[u] = xqr[u] = xpi[u] = xqi[u] = 0.0;
      if (u < urows) {
        xpr[u] = M.ld(gpr + i);
        xqr[u] = M.ld(gqr + i);
        if (CPLX) {
          xpi[u] = M.ld(gpi + i);
          xqi[u] = M.ld(gqi + i);
        }
      }
    }
    if (rk) {  // section 3.2, step 2: both columns downscaled by 2^rk first
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u < urows) {
          xpr[u] = ldexp_rn(xpr[u], rk);
          xqr[u] = ldexp_rn(xqr[u], rk);
          if (CPLX) {
            xpi[u] = ldexp_rn(xpi[u], rk);
            xqi[u] = ldexp_rn(xqi[u], rk);
          }
          if ((u & (kGroupWarps - 1)) == g) {  // each row stored by one warp
            const int i = lane + 32 * u;
            M.st(gpr + i, xpr[u]);
            M.st(gqr + i, xqr[u]);
            if (CPLX) {
              M.st(gpi + i, xpi[u]);
              M.st(gqi + i, xqi[u]);
            }
          }
        }
      }
    }
    // this warp's sum, the rows in ascending order as pair_sums forms it:
    //   g = 0: xpr xpr (+ xpi xpi)     g = 1: xqr xqr (+ xqi xqi)
    //   g = 2: xqr xpr (+ xqi xpi)     g = 3: xqr xpi + (-xqi) xpr (complex)
    // with the operands picked by selects, so that the loop has no branch
    // (a real pair's warp 3 forms a sum nobody reads)
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (u < urows) {
        const double a1 = (g == 0) ? xpr[u] : xqr[u];
        const double b1 = (g == 0 || g == 2) ? xpr[u] : (g == 1) ? xqr[u] : xpi[u];
        acc = __fma_rn(a1, b1, acc);
        if (CPLX) {
          const double a2 = (g == 0) ? xpi[u] : (g == 3) ? dbl(bits(xqi[u]) ^ kSign) : xqi[u];
          const double b2 = (g == 0 || g == 2) ? xpi[u] : (g == 1) ? xqi[u] : xpr[u];
          acc = __fma_rn(a2, b2, acc);
        }
      }
    }
    if (CPLX || g < 3) {
      acc = warp_sum(acc);
      if (lane == 0) s_sum[g] = acc;
    }
    __syncthreads();
    PairSums sm;
    sm.pp = s_sum[0];
    sm.qq = s_sum[1];
    sm.qr = s_sum[2];
    sm.qi = CPLX ? s_sum[3] : 0.0;
    sm.fp = sm.fq = 1.0;
    sm.ep = sm.eq = 0;
    sm.wide = 0;
    __syncthreads();  // s_sum is free for the next pair
    // squares below 2^-1022 may have lost bits: the wide-exponent sums
    // (every warp the same, from the columns as stored)
    if (bits(sm.pp) < kWideBelow || bits(sm.qq) < kWideBelow) {
      sm = pair_sums_wide<CPLX, CG, false>(M, p, q);
      __syncthreads();  // every warp has read the columns before any writes them
    }
    if (gv.p >= 0) gv.load(M, g);  // the last step's V rows, in flight during the rotation
    PairOut o = pair_rotation_warp<CPLX>(sm, ups);
    o.swap = o.swap && permute;
    if (gv.p >= 0) gv.apply(M, g);
    double *dpr = o.swap ? gqr : gpr, *dqr = o.swap ? gpr : gqr;
    double *dpi = o.swap ? gqi : gpi, *dqi = o.swap ? gpi : gqi;
    if (o.rot && o.gs) {  // Eq. e:GS replaces the rotation on G: one warp
      if (g == 0) gs_apply<CPLX, CG>(M, p, q, o, Mloc);
    } else if (o.rot || o.swap) {
      // warp g's rows u = g + 4 j, picked from the registers by selects
      // (no branch per row); a swap without rotation stores the rows as
      // they are
#pragma unroll
      for (int j = 0; j < U / kGroupWarps; ++j) {
        const int u0 = kGroupWarps * j, u = u0 + g;
        double pr = xpr[u0], pi = xpi[u0], qr = xqr[u0], qi = xqi[u0];
#pragma unroll
        for (int t = 1; t < kGroupWarps; ++t) {
          pr = (g == t) ? xpr[u0 + t] : pr;
          qr = (g == t) ? xqr[u0 + t] : qr;
          if (CPLX) {
            pi = (g == t) ? xpi[u0 + t] : pi;
            qi = (g == t) ? xqi[u0 + t] : qi;
          }
        }
        if (u < urows) {
          const int i = lane + 32 * u;
          double npr, npi, nqr, nqi;
          rotate_row<double, CPLX>(pr, pi, qr, qi, o.c, o.C, o.S, npr, npi, nqr, nqi);
          unsigned long long mr = max(magbits(npr), magbits(nqr));
          if (CPLX) mr = max(mr, max(magbits(npi), magbits(nqi)));
          Mloc = o.rot ? max(Mloc, mr) : Mloc;
          M.st(dpr + i, o.rot ? npr : pr);
          M.st(dqr + i, o.rot ? nqr : qr);
          if (CPLX) {
            M.st(dpi + i, o.rot ? npi : pi);
            M.st(dqi + i, o.rot ? nqi : qi);
          }
        }
      }
    }
    if (o.rot || o.swap) {
      gv.p = p;
      gv.q = q;
      gv.o = o;
    }
    if (g == 0 && lane == 0) {
      if (o.rot) ++rots;
      if (o.gs) ++gsn;
    }
  }
}

// GW = 2 or 4 warps of a block on each pair for long columns (step_group
// keeps a pair's rows in registers; here they stream through in trips of U
// rows per lane).  Warp g forms the sums s = g, g + GW, ... of (0 ||g_p||^2,
// 1 ||g_q||^2, 2 Re g_q^* g_p, 3 Im g_q^* g_p) over all the rows, each in
// the canonical lane order (lane l: rows l, l + 32, ... ascending), as
// pair_sums forms that sum, and reduces each by warp_sum; every warp
// computes the rotation; the transformation of G's and then V's rows is
// shared out by trips, warp g taking trips g, g + GW, ...  A warp's FP64 (or
// FP32) instruction stream per step is then about 1/GW of the one-warp
// form's, and GW times as many warps keep the SM's pipes and memory busy.
// The same sums, rotations and transformed rows, so the same bits.  lastmod
// etc.: as in step_warps.
template <typename T, bool CPLX, int CG, int GW>
__device__ __forceinline__ void step_group_stream(const MatViewT<T, CG> &M, int k, int nt, double ups,
                                                  int rk, bool permute, unsigned long long &Mloc,
                                                  int &rots, int &gsn, double *s_sum, int *lastmod,
                                                  int gstep, int last_rescale)
{
  static_assert(GW == 2 || GW == 4, "2 or 4 warps per pair");
  constexpr int U = (sizeof(T) == 4) ? 8 : 4;  // rows per lane per trip
  constexpr int NS = 4 / GW;                    // sums per warp
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int L = nt / 2, K = nt - 1;
  const int nsum = CPLX ? 4 : 3;
  for (int l = blockIdx.x; l < L; l += gridDim.x) {
    int p, q;
    pair_of(k, l, nt, p, q);
    if (q >= M.n) {
      if (rk && g == 0) {  // phantom partner: only a pending rescale applies
        scale_col(M, M.Gr(p), rk, lane);
        if (CPLX) scale_col(M, M.Gi(p), rk, lane);
      }
      continue;
    }
    if (lastmod != nullptr && rk == 0 && gstep - K > last_rescale) {
      const int before = gstep - K;  // the pair's last meeting, one sweep ago
      if (__ldcg(lastmod + p) < before && __ldcg(lastmod + q) < before) continue;
    }
    T *gpr = M.Gr(p), *gqr = M.Gr(q);
    T *gpi = CPLX ? M.Gi(p) : nullptr, *gqi = CPLX ? M.Gi(q) : nullptr;
    if (rk) {  // section 3.2, step 2: both columns downscaled by 2^rk, trips shared out
      for (int base = lane + 32 * U * g; base < M.mp; base += 32 * U * GW) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = base + 32 * u;
          if (i < M.mp) {
            M.st(gpr + i, ldexp_rn(M.ld(gpr + i), rk));
            M.st(gqr + i, ldexp_rn(M.ld(gqr + i), rk));
            if (CPLX) {
              M.st(gpi + i, ldexp_rn(M.ld(gpi + i), rk));
              M.st(gqi + i, ldexp_rn(M.ld(gqi + i), rk));
            }
          }
        }
      }
      __syncthreads();  // every row scaled before any warp sums
    }
    // this warp's sums; it loads only the planes they read (sum 0: g_p,
    // 1: g_q, 2 and 3: both)
    const bool need_p = GW == 2 || g != 1, need_q = GW == 2 || g != 0;
    T acc[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) acc[j] = T(0);
    if (g < nsum) {
      for (int base = lane; base < M.mp; base += 32 * U) {
        T xpr[U], xqr[U], xpi[U], xqi[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = base + 32 * u;
          xpr[u] = xqr[u] = xpi[u] = xqi[u] = T(0);
          if (i < M.mp) {
            if (need_p) {
              xpr[u] = M.ld(gpr + i);
              if (CPLX) xpi[u] = M.ld(gpi + i);
            }
            if (need_q) {
              xqr[u] = M.ld(gqr + i);
              if (CPLX) xqi[u] = M.ld(gqi + i);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (base + 32 * u < M.mp) {
#pragma unroll
            for (int j = 0; j < NS; ++j) {
              const int sidx = g + GW * j;
              if (sidx == 0) {
                acc[j] = fma_t(xpr[u], xpr[u], acc[j]);
                if (CPLX) acc[j] = fma_t(xpi[u], xpi[u], acc[j]);
              } else if (sidx == 1) {
                acc[j] = fma_t(xqr[u], xqr[u], acc[j]);
                if (CPLX) acc[j] = fma_t(xqi[u], xqi[u], acc[j]);
              } else if (sidx == 2) {
                acc[j] = fma_t(xqr[u], xpr[u], acc[j]);
                if (CPLX) acc[j] = fma_t(xqi[u], xpi[u], acc[j]);
              } else if (CPLX) {
                acc[j] = fma_t(xqr[u], xpi[u], acc[j]);
                acc[j] = fma_t(-xqi[u], xpr[u], acc[j]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const int sidx = g + GW * j;
        if (sidx < nsum) {
          const double tot = warp_sum((double)acc[j]);
          if (lane == 0) s_sum[sidx] = tot;
        }
      }
    }
    __syncthreads();
    PairSums sm;
    sm.pp = s_sum[0];
    sm.qq = s_sum[1];
    sm.qr = s_sum[2];
    sm.qi = CPLX ? s_sum[3] : 0.0;
    sm.fp = sm.fq = 1.0;
    sm.ep = sm.eq = 0;
    sm.wide = 0;
    __syncthreads();  // s_sum is free for the next pair
    if constexpr (sizeof(T) == 8) {
      // squares below 2^-1022 may have lost bits: the wide-exponent sums
      if (bits(sm.pp) < kWideBelow || bits(sm.qq) < kWideBelow) {
        sm = pair_sums_wide<CPLX, CG, false>(M, p, q);
        __syncthreads();  // every warp has read the columns before any writes them
      }
    }
    PairOut o = pair_rotation_warp<CPLX>(sm, ups);
    o.swap = o.swap && permute;
    if (o.rot || o.swap) {
      const T c = to_t(o.c, T(0)), C = to_t(o.C, T(0));
      const T S = CPLX ? to_t(o.S, T(0)) : T(0);
      bool gdone = false;
      if constexpr (sizeof(T) == 8) {
        if (o.rot && o.gs) {  // Eq. e:GS replaces the rotation on G: one warp
          if (g == 0) gs_apply<CPLX, CG>(M, p, q, o, Mloc);
          gdone = true;
        }
      }
      for (int pass = gdone ? 1 : 0; pass < 2; ++pass) {
        const bool onG = (pass == 0);
        const int rows = onG ? M.mp : M.np;
        T *xpr = onG ? gpr : M.Vr(p), *xqr = onG ? gqr : M.Vr(q);
        T *xpi = CPLX ? (onG ? gpi : M.Vi(p)) : nullptr;
        T *xqi = CPLX ? (onG ? gqi : M.Vi(q)) : nullptr;
        T *dpr = o.swap ? xqr : xpr, *dqr = o.swap ? xpr : xqr;
        T *dpi = o.swap ? xqi : xpi, *dqi = o.swap ? xpi : xqi;
        for (int base = lane + 32 * U * g; base < rows; base += 32 * U * GW) {
          T pr[U], qr[U], pi[U], qi[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = base + 32 * u;
            pr[u] = qr[u] = pi[u] = qi[u] = T(0);
            if (i < rows) {
              pr[u] = M.ld(xpr + i);
              qr[u] = M.ld(xqr + i);
              if (CPLX) {
                pi[u] = M.ld(xpi + i);
                qi[u] = M.ld(xqi + i);
              }
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = base + 32 * u;
            if (i < rows) {
              T npr = pr[u], npi = pi[u], nqr = qr[u], nqi = qi[u];
              if (o.rot) {
                rotate_row<T, CPLX>(pr[u], pi[u], qr[u], qi[u], c, C, S, npr, npi, nqr, nqi);
                if (onG) {
                  Mloc = max(Mloc, max(magbits(npr), magbits(nqr)));
                  if (CPLX) Mloc = max(Mloc, max(magbits(npi), magbits(nqi)));
                }
              }
              M.st(dpr + i, npr);
              M.st(dqr + i, nqr);
              if (CPLX) {
                M.st(dpi + i, npi);
                M.st(dqi + i, nqi);
              }
            }
          }
        }
      }
    }
    if (g == 0 && lane == 0) {
      if (o.rot) ++rots;
      if (o.gs) ++gsn;
      if (lastmod != nullptr && (o.rot || o.swap)) {
        __stcg(lastmod + p, gstep);
        __stcg(lastmod + q, gstep);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Finalisation pieces (section 4.2.1), shared by the single-matrix and the
// batched kernels so that both produce the same bits.

// Column j's norm as (e, f) by one warp in the canonical order (the
// wide-exponent norm when the plain sum of squares is too small to trust);
// a zero column gets e = INT_MIN, f = 1.
template <bool CPLX, int CG>
__device__ __forceinline__ void colnorm_warp(const MatViewT<double, CG> &M, int j, int lane, int *e_out,
                                             double *f_out)
{
  const double *xr = M.Gr(j), *xi = CPLX ? M.Gi(j) : nullptr;
  double s = 0.0;
  for (int i = lane; i < M.mp; i += 32) {
    const double a = M.ld(xr + i);
    s = __fma_rn(a, a, s);
    if (CPLX) {
      const double b = M.ld(xi + i);
      s = __fma_rn(b, b, s);
    }
  }
  s = warp_sum(s);
  if (bits(s) < kWideBelow) {
    // squares may have fallen below the normal range: the wide-exponent
    // norm (Alg. rnF) instead (kNegInfE == INT_MIN marks a zero column)
    EF r = {kNegInfE, 1.0};
    for (int i = lane; i < M.mp; i += 32) {
      ef_fma_step(M.ld(xr + i), r);
      if (CPLX) ef_fma_step(M.ld(xi + i), r);
    }
    r = ef_sqrt(ef_warp_sum(r));
    if (lane == 0) {
      e_out[j] = r.e;
      f_out[j] = r.f;
    }
    return;
  }
  if (lane == 0) {
    const double r = __dsqrt_rn(s);
    const int e = flg(r);
    e_out[j] = e;
    f_out[j] = ldexp_rn(r, -e);
  }
}

__device__ __forceinline__ bool ef_less(int ea, double fa, int eb, double fb)
{
  return (ea != eb) ? (ea < eb) : (bits(fa) < bits(fb));
}

// Position of column j after a stable sort by non-increasing sigma:
// #{i : sigma_i > sigma_j, or sigma_i == sigma_j and i < j}.
__device__ __forceinline__ int rank_of(int n, const int *e, const double *f, int j)
{
  int r = 0;
  const int ej = e[j];
  const double fj = f[j];
  for (int i = 0; i < n; ++i) {
    const int ei = e[i];
    const double fi = f[i];
    const bool gt = ef_less(ej, fj, ei, fi);
    const bool eq = (ei == ej) && (bits(fi) == bits(fj));
    r += (gt || (eq && i < j)) ? 1 : 0;
  }
  return r;
}

// One element (row i) of output column j, which goes to position r:
// U(i, r) = G(i, j) 2^{-e_j} / f_j (i < m), V(i, r) = V_k(i, j) (i < n).
template <bool CPLX, int CG>
__device__ __forceinline__ void output_elem(const MatViewT<double, CG> &M, int i, int j, int r, int ej,
                                            double fj, bool bad, double *U, int64_t ldu,
                                            double *V, int64_t ldv)
{
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const bool zero = (ej == INT_MIN);
  if (i < M.m) {
    double ur = 0.0, ui = 0.0;
    if (bad) {
      ur = ui = nan;
    } else if (!zero) {
      ur = __ddiv_rn(ldexp_rn(M.ld(M.Gr(j) + i), -ej), fj);
      if (CPLX) ui = __ddiv_rn(ldexp_rn(M.ld(M.Gi(j) + i), -ej), fj);
    }
    if (CPLX) {
      U[2 * (r * ldu + i)] = ur;
      U[2 * (r * ldu + i) + 1] = ui;
    } else {
      U[r * ldu + i] = ur;
    }
  }
  if (i < M.n) {
    const double vr = bad ? nan : M.ld(M.Vr(j) + i);
    if (CPLX) {
      V[2 * (r * ldv + i)] = vr;
      V[2 * (r * ldv + i) + 1] = bad ? nan : M.ld(M.Vi(j) + i);
    } else {
      V[r * ldv + i] = vr;
    }
  }
}

// sigma_r = 2^{e_j - s} f_j and its (e, f) pair.
__device__ __forceinline__ void output_sigma(int r, int ej, double fj, int s, bool bad,
                                             double *sigma, double *sigma_e, double *sigma_f)
{
  const double nan = __longlong_as_double(0x7FF8000000000000ll);
  const bool zero = (ej == INT_MIN);
  if (sigma) sigma[r] = bad ? nan : zero ? 0.0 : ldexp_rn(fj, ej - s);
  if (sigma_e)
    sigma_e[r] = bad ? nan : zero ? -__longlong_as_double((long long)kInf) : (double)(ej - s);
  if (sigma_f) sigma_f[r] = bad ? nan : fj;
}

// Device-wide time in ns (for bounded waits).
__device__ __forceinline__ unsigned long long global_ns()
{
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier for a cooperative (co-resident) launch, one reduction per
// block: block 0 adds 2^31 - (gridDim.x - 1) to *word and every other
// block 1, so the top bit of *word flips exactly when the last block
// arrives (the partial sums stay below 2^31 past the value at the start),
// and each block waits until the top bit differs from the phase it holds.
// A block already at the next barrier cannot flip the bit back before every
// block has left this one.  Thread 0 of each block keeps that phase: read
// once before its first arrival (barrier_phase; the bit cannot flip before
// every block has arrived) and toggled at each barrier, so the arrival is a
// reduction that returns nothing (red.release.gpu: the block's writes,
// ordered before it by the block barrier, are released with it) and the
// wait polls with acquire loads (ld.acquire.gpu), with no full fences.
// The wait is bounded: after limit_ns (or once another block has reported
// a timeout in *err, read every 64 polls) it sets *err = 1 and returns
// false, so a lost block can never hang the GPU; callers then leave the
// kernel.  The low 31 bits of *word must be 0 at launch.
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned int *p, unsigned int v)
{
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The phase thread 0 starts with: call before the block's first arrival.
__device__ __forceinline__ unsigned int barrier_phase(const unsigned int *word)
{
  return (threadIdx.x == 0) ? (*(const volatile unsigned int *)word >> 31) : 0u;
}

__device__ __forceinline__ bool grid_barrier(unsigned int *word, volatile int *err,
                                             unsigned long long limit_ns, unsigned int &phase)
{
  __shared__ int s_fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int add = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1u)) : 1u;
    red_release_gpu_add(word, add);
    int fail = 0;
    const unsigned long long t0 = global_ns();
    for (unsigned int it = 1; (ld_acquire_gpu(word) >> 31) == phase; ++it) {
      if ((it & 63u) == 0u && (*err || global_ns() - t0 > limit_ns)) {
        *err = 1;
        fail = 1;
        break;
      }
    }
    phase ^= 1u;
    s_fail = fail;
  }
  __syncthreads();
  return s_fail == 0;
}

}  // namespace jsvd

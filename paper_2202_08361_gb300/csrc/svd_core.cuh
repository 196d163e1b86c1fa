// svd_core.cuh -- one warp, one pivot pair: the fused step of the one-sided
// Jacobi SVD (Alg. zvjsvd, lines spade..star), shared by the single-matrix
// persistent kernel and the batched kernel.
//
// The warp reads the pair's columns once for the three sums, reduces them
// in a canonical order (lane l accumulates rows l, l+32, l+64, ... in
// ascending order with fma, then an xor butterfly over offsets 16, 8, 4, 2,
// 1), so the bits never depend on the launch shape.  Lane 0 forms the (e,f)
// norms, the scaled dot-product (Alg. zdpscl semantics: power-of-two
// prescaling, one final division by f_q f_p), the convergence test
// (Eq. e:tol, Alg. cvg), the scaled Grammian (Alg. Gram) and its 2x2 EVD,
// and broadcasts the rotation; the whole warp then applies Eq. e:transf
// (Alg. zjrot) to the G and V column pairs, swapping per the permutation
// bit, and tracks the max-norm of the new G columns (section 3.2, step 4).
#pragma once
#include "evd2.cuh"

namespace jsvd {

// Loads and stores of G and V inside the persistent kernels bypass L1: a
// column written by another SM in the previous step must not be served from
// a stale L1 line (L1 is not coherent across SMs; the grid barrier only
// orders L2).
__device__ __forceinline__ double ldg2(const double *p) { return __ldcg(p); }
__device__ __forceinline__ void stg2(double *p, double v) { __stcg(p, v); }

struct MatView {
  double *gr, *gi;   // G planes (gi == nullptr for real), column j at + j*ldg
  double *vr, *vi;   // V planes, column j at + j*ldv
  int m, n;          // true sizes
  int mp, np;        // rows padded to a multiple of 32 (padding rows are 0)
  int64_t ldg, ldv;
};

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

__device__ __forceinline__ unsigned long long warp_umax(unsigned long long x)
{
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = (y > x) ? y : x;
  }
  return x;
}

// |x| bits of a finite double: ordered like the magnitudes
__device__ __forceinline__ unsigned long long abits(double x) { return bits(x) & ~kSign; }

// Alg. hypot (naive, reproducible)
__device__ __forceinline__ double hypot_naive(double x, double y)
{
  const double ax = dabs(x), ay = dabs(y);
  const bool xm = bits(ax) <= bits(ay);
  const double m = xm ? ax : ay, M = xm ? ay : ax;
  const double q = (bits(M) == 0ull) ? 0.0 : __ddiv_rn(m, M);
  return __dmul_rn(__dsqrt_rn(__fma_rn(q, q, 1.0)), M);
}

// Scale a column by 2^k in place (rows < mp).
__device__ __forceinline__ void scale_col(double *x, int mp, int k, int lane)
{
  for (int i = lane; i < mp; i += 32) stg2(x + i, ldexp_rn(ldg2(x + i), k));
}

struct PairOut {
  bool rot, swap;
  double c, C, S;
};

// Lane-0 part: from the sums to the rotation (Alg. zdpscl's division,
// Alg. cvg, Alg. Gram, the EVD).  spp = ||g_p||^2, sqq = ||g_q||^2,
// (sqr, sqi) = g_q^* g_p, all of the current (scaled) G.
template <bool CPLX>
__device__ __forceinline__ PairOut pair_rotation(double spp, double sqq, double sqr, double sqi,
                                                 double ups)
{
  PairOut o;
  o.c = 1.0;
  o.C = 0.0;
  o.S = 0.0;
  if (bits(spp) == 0ull || bits(sqq) == 0ull) {
    // a zero column: never rotated; swapped iff ||g_p|| < ||g_q||
    o.rot = false;
    o.swap = bits(spp) < bits(sqq);
    return o;
  }
  // (e,f) norms: ||g_j|| = 2^e_j f_j, 1 <= f_j < 2
  const double rp = __dsqrt_rn(spp), rq = __dsqrt_rn(sqq);
  const int ep = flg(rp), eq = flg(rq);
  const double fp = ldexp_rn(rp, -ep), fq = ldexp_rn(rq, -eq);
  // a21' = (g_q/2^eq)^* (g_p/2^ep) / (f_q f_p)
  const double d = __dmul_rn(fq, fp);
  const double zr = __ddiv_rn(ldexp_rn(sqr, -(ep + eq)), d);
  const double zi = CPLX ? __ddiv_rn(ldexp_rn(sqi, -(ep + eq)), d) : 0.0;
  const double az = CPLX ? hypot_naive(zr, zi) : dabs(zr);
  o.rot = !(ord(az) < ord(ups));
  // Alg. Gram
  double f12 = __ddiv_rn(fp, fq), f21 = __ddiv_rn(fq, fp);
  int e12 = ep - eq + flg(f12), e21 = eq - ep + flg(f21);
  f12 = ldexp_rn(f12, -flg(f12));
  f21 = ldexp_rn(f21, -flg(f21));
  const int sA = min(1023 - max(e12, e21), 0);
  const double b11 = ldexp_rn(f12, e12 + sA), b22 = ldexp_rn(f21, e21 + sA);
  const double b21r = ldexp_rn(zr, sA);
  Rot2 r;
  if (CPLX) {
    r = zsjac2(b11, b22, b21r, ldexp_rn(zi, sA));
  } else {
    r = dsjac2(b11, b22, b21r);
  }
  o.swap = perm_bit(r) != 0;
  o.c = r.cphi;
  o.C = r.etr;
  o.S = r.eti;
  return o;
}

// The fused step for pair (p, q), executed by one full warp.  rk != 0
// downscales both columns of G by 2^rk first (section 3.2, step 2);
// permute applies the column swap P.
// Returns (in lane 0) whether the pair was rotated; Mloc collects the
// magnitude bits of the transformed G entries.
template <bool CPLX>
__device__ __forceinline__ bool pair_step(const MatView &M, int p, int q, double ups, int rk,
                                          bool permute, unsigned long long &Mloc)
{
  const int lane = threadIdx.x & 31;
  double *gpr = M.gr + p * M.ldg, *gqr = M.gr + q * M.ldg;
  double *gpi = CPLX ? M.gi + p * M.ldg : nullptr, *gqi = CPLX ? M.gi + q * M.ldg : nullptr;
  double spp = 0.0, sqq = 0.0, sqr = 0.0, sqi = 0.0;
  for (int i = lane; i < M.mp; i += 32) {
    double xpr = ldg2(gpr + i), xqr = ldg2(gqr + i);
    double xpi = 0.0, xqi = 0.0;
    if (CPLX) {
      xpi = ldg2(gpi + i);
      xqi = ldg2(gqi + i);
    }
    if (rk) {
      xpr = ldexp_rn(xpr, rk);
      xqr = ldexp_rn(xqr, rk);
      stg2(gpr + i, xpr);
      stg2(gqr + i, xqr);
      if (CPLX) {
        xpi = ldexp_rn(xpi, rk);
        xqi = ldexp_rn(xqi, rk);
        stg2(gpi + i, xpi);
        stg2(gqi + i, xqi);
      }
    }
    spp = __fma_rn(xpr, xpr, spp);
    sqq = __fma_rn(xqr, xqr, sqq);
    sqr = __fma_rn(xqr, xpr, sqr);
    if (CPLX) {
      spp = __fma_rn(xpi, xpi, spp);
      sqq = __fma_rn(xqi, xqi, sqq);
      sqi = __fma_rn(xqr, xpi, sqi);
      sqr = __fma_rn(xqi, xpi, sqr);
      sqi = __fma_rn(-xqi, xpr, sqi);
    }
  }
  spp = warp_sum(spp);
  sqq = warp_sum(sqq);
  sqr = warp_sum(sqr);
  if (CPLX) sqi = warp_sum(sqi);
  PairOut o = {};
  if (lane == 0) {
    o = pair_rotation<CPLX>(spp, sqq, sqr, sqi, ups);
    o.swap = o.swap && permute;
  }
  const unsigned full = 0xffffffffu;
  const int flags = __shfl_sync(full, lane == 0 ? ((o.rot ? 1 : 0) | (o.swap ? 2 : 0)) : 0, 0);
  const bool rot = flags & 1, swp = (flags >> 1) & 1;
  if (rot) {
    const double c = __shfl_sync(full, o.c, 0), C = __shfl_sync(full, o.C, 0);
    const double S = CPLX ? __shfl_sync(full, o.S, 0) : 0.0;
    double *dpr = swp ? gqr : gpr, *dqr = swp ? gpr : gqr;
    double *dpi = swp ? gqi : gpi, *dqi = swp ? gpi : gqi;
    // Eq. e:transf on G: g_p' = fma(g_q, e', g_p) c, g_q' = fma(g_p, -conj(e'), g_q) c
    for (int i = lane; i < M.mp; i += 32) {
      const double pr = ldg2(gpr + i), qr = ldg2(gqr + i);
      if (CPLX) {
        const double pi = ldg2(gpi + i), qi = ldg2(gqi + i);
        const double npr = __dmul_rn(__fma_rn(qr, C, __fma_rn(-qi, S, pr)), c);
        const double npi = __dmul_rn(__fma_rn(qr, S, __fma_rn(qi, C, pi)), c);
        const double nqr = __dmul_rn(__fma_rn(pr, -C, __fma_rn(-pi, S, qr)), c);
        const double nqi = __dmul_rn(__fma_rn(pr, S, __fma_rn(pi, -C, qi)), c);
        stg2(dpr + i, npr);
        stg2(dpi + i, npi);
        stg2(dqr + i, nqr);
        stg2(dqi + i, nqi);
        unsigned long long a = max(max(abits(npr), abits(npi)), max(abits(nqr), abits(nqi)));
        Mloc = max(Mloc, a);
      } else {
        const double npr = __dmul_rn(__fma_rn(qr, C, pr), c);
        const double nqr = __dmul_rn(__fma_rn(pr, -C, qr), c);
        stg2(dpr + i, npr);
        stg2(dqr + i, nqr);
        Mloc = max(Mloc, max(abits(npr), abits(nqr)));
      }
    }
    double *vpr = M.vr + p * M.ldv, *vqr = M.vr + q * M.ldv;
    double *vpi = CPLX ? M.vi + p * M.ldv : nullptr, *vqi = CPLX ? M.vi + q * M.ldv : nullptr;
    double *wpr = swp ? vqr : vpr, *wqr = swp ? vpr : vqr;
    double *wpi = swp ? vqi : vpi, *wqi = swp ? vpi : vqi;
    for (int i = lane; i < M.np; i += 32) {
      const double pr = ldg2(vpr + i), qr = ldg2(vqr + i);
      if (CPLX) {
        const double pi = ldg2(vpi + i), qi = ldg2(vqi + i);
        const double npr = __dmul_rn(__fma_rn(qr, C, __fma_rn(-qi, S, pr)), c);
        const double npi = __dmul_rn(__fma_rn(qr, S, __fma_rn(qi, C, pi)), c);
        const double nqr = __dmul_rn(__fma_rn(pr, -C, __fma_rn(-pi, S, qr)), c);
        const double nqi = __dmul_rn(__fma_rn(pr, S, __fma_rn(pi, -C, qi)), c);
        stg2(wpr + i, npr);
        stg2(wpi + i, npi);
        stg2(wqr + i, nqr);
        stg2(wqi + i, nqi);
      } else {
        const double npr = __dmul_rn(__fma_rn(qr, C, pr), c);
        const double nqr = __dmul_rn(__fma_rn(pr, -C, qr), c);
        stg2(wpr + i, npr);
        stg2(wqr + i, nqr);
      }
    }
  } else if (swp) {
    for (int i = lane; i < M.mp; i += 32) {
      const double a = ldg2(gpr + i), b = ldg2(gqr + i);
      stg2(gpr + i, b);
      stg2(gqr + i, a);
      if (CPLX) {
        const double ai = ldg2(gpi + i), bi = ldg2(gqi + i);
        stg2(gpi + i, bi);
        stg2(gqi + i, ai);
      }
    }
    double *vpr = M.vr + p * M.ldv, *vqr = M.vr + q * M.ldv;
    for (int i = lane; i < M.np; i += 32) {
      const double a = ldg2(vpr + i), b = ldg2(vqr + i);
      stg2(vpr + i, b);
      stg2(vqr + i, a);
      if (CPLX) {
        double *vpi = M.vi + p * M.ldv, *vqi = M.vi + q * M.ldv;
        const double ai = ldg2(vpi + i), bi = ldg2(vqi + i);
        stg2(vpi + i, bi);
        stg2(vqi + i, ai);
      }
    }
  }
  __syncwarp();
  return rot;
}

// Device-wide time in ns (for bounded waits).
__device__ __forceinline__ unsigned long long global_ns()
{
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sense-reversing grid barrier for a cooperative (co-resident) launch.
// The wait is bounded: after limit_ns it sets *err = 1 and returns, so a
// lost block can never hang the GPU; callers then leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned int *count, volatile unsigned int *gen,
                                             volatile int *err, unsigned long long limit_ns)
{
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int arrived = atomicAdd(count, 1u) + 1u;
    if (arrived == gridDim.x) {
      *count = 0u;
      __threadfence();
      atomicAdd((unsigned int *)gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*err) break;
        if (global_ns() - t0 > limit_ns) {
          *err = 1;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *err == 0;
}

}  // namespace jsvd

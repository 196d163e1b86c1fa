// svd.cu -- jsvd_svd: the one-sided Jacobi SVD of one matrix (Alg. zvjsvd).
//
// Phases (one stream, no host synchronisation):
//   1. maxnorm_kernel   M~_0 = ||A||_max (NaN -> Inf), section 3.2
//   2. init_kernel      G_1 = 2^{s_0} A split into planes, V_1 = I
//   3. sweeps_kernel    persistent cooperative kernel: every sweep, every
//                       step, one warp per pivot pair (svd_core.cuh: sums,
//                       rotation, transformation), a bounded grid barrier
//                       between steps, stop on a rotation-free sweep
//   4. colnorm_kernel   final (e,f) norms of the columns
//   5. rank_kernel      stable non-increasing order of sigma, info
//   6. output_kernel    U = G 2^{-e_j} / f_j, V, sigma, merged planes
//
// Scaling (section 3.2, adapted): the paper keeps ||G||_max below
// nu/(varsigma m) so that an xNRM2-style norm cannot overflow.  Here the
// three sums of a pair are formed in one pass as plain sums of squares and
// products, which is safe while the entries stay below 2^rescale_exp (the
// safe region of supplement SM3; 2^480 by default): G_1 is scaled to a
// max-norm in [2^(R-25), 2^(R-24)), R = rescale_exp, and scaled back there
// whenever the tracked max-norm M~ reaches 2^R.  The high binade leaves tiny
// columns the most room above the subnormal range; columns whose squares
// still fall below it take the wide-exponent norms (Alg. rnF).
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "jsvd_internal.h"
#include "svd_core.cuh"

namespace jsvd {

constexpr int kMaxSweepsCap = 4096;
constexpr unsigned long long kBarrierLimitNs = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s

// Device-side state at the start of the workspace.
struct SvdState {
  unsigned long long Mbuf[3];  // running max-norm (bits), triple-buffered by step
  unsigned long long M0;       // ||A||_max bits
  unsigned int bar_word;        // grid barrier (low 31 bits 0 at launch)
  int err;                     // barrier timeout
  int nonfinite;
  int s;                       // accumulated scaling exponent: G = 2^s (A V)
  int rescales;
  int sweeps;
  int converged;
  int T[kMaxSweepsCap];        // transformations per sweep
  unsigned long long gs;       // Gram-Schmidt steps (Eq. e:GS) in all
};

struct SvdLayout {
  size_t state, gr, gi, vr, vi, e, f, rank, total;
  int mp, np;
  int64_t ldg, ldv;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static SvdLayout svd_layout(bool cplx, int64_t m, int64_t n)
{
  SvdLayout L;
  L.mp = (int)((m + 31) / 32 * 32);
  L.np = (int)((n + 31) / 32 * 32);
  L.ldg = L.mp;
  L.ldv = L.np;
  size_t o = 0;
  L.state = o;
  o = align256(o + sizeof(SvdState));
  L.gr = o;
  o = align256(o + sizeof(double) * (size_t)L.ldg * (size_t)n);
  L.gi = o;
  if (cplx) o = align256(o + sizeof(double) * (size_t)L.ldg * (size_t)n);
  L.vr = o;
  o = align256(o + sizeof(double) * (size_t)L.ldv * (size_t)n);
  L.vi = o;
  if (cplx) o = align256(o + sizeof(double) * (size_t)L.ldv * (size_t)n);
  L.e = o;
  o = align256(o + sizeof(int) * (size_t)n);
  L.f = o;
  o = align256(o + sizeof(double) * (size_t)n);
  L.rank = o;
  o = align256(o + sizeof(int) * (size_t)n);
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------

// max over count doubles of |x| with NaN -> Inf, as ordered bits
__global__ void maxnorm_kernel(const double *__restrict__ A, int64_t lda, int64_t rows, int64_t cols,
                               unsigned long long *out)
{
  unsigned long long mx = 0ull;
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / rows, i = t - j * rows;
    unsigned long long a = abits(A[j * lda + i]);
    a = (a > kInf) ? kInf : a;  // min(|y|, Inf): NaN -> Inf
    mx = (a > mx) ? a : mx;
  }
  mx = warp_umax(mx);
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// G_1 = 2^{s_0} A (planes), V_1 = I; s_0 brings ||A||_max into
// [2^target, 2^(target + 1)).  Complex A is interleaved: plane r takes the
// even doubles, plane i the odd.
template <bool CPLX>
__global__ void init_kernel(const double *__restrict__ A, int64_t lda, MatView M, SvdState *st,
                            int target)
{
  const unsigned long long m0 = st->M0;
  const bool nonfinite = m0 >= kInf;
  const int s0 = (m0 == 0ull || nonfinite) ? 0 : target - flg(dbl(m0));
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    st->s = s0;
    st->nonfinite = nonfinite ? 1 : 0;
    st->Mbuf[0] = (m0 == 0ull || nonfinite) ? 0ull : bits(ldexp_rn(dbl(m0), s0));
  }
  for (int j = blockIdx.y; j < M.n; j += gridDim.y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M.mp, M.np);
         i += gridDim.x * blockDim.x) {
      if (i < M.mp) {
        double xr = 0.0, xi = 0.0;
        if (i < M.m && !nonfinite) {
          if (CPLX) {
            xr = ldexp_rn(A[2 * (j * lda + i)], s0);
            xi = ldexp_rn(A[2 * (j * lda + i) + 1], s0);
          } else {
            xr = ldexp_rn(A[j * lda + i], s0);
          }
        }
        M.gr[j * M.ldg + i] = xr;
        if (CPLX) M.gi[j * M.ldg + i] = xi;
      }
      if (i < M.np) {
        M.vr[j * M.ldv + i] = (i == j) ? 1.0 : 0.0;
        if (CPLX) M.vi[j * M.ldv + i] = 0.0;
      }
    }
  }
}

// All sweeps of Alg. zvjsvd in one cooperative launch; the blocks stride
// over the nt/2 pairs of a step and a bounded grid barrier separates the
// steps.  Two forms of a block's share of a step, with the same bits:
//   kFlagWarpStep (the default): each warp runs its pairs alone (sums,
//     rotation spread over the warp's lanes, transformation), no block
//     barrier inside a step;
//   otherwise chunks of W pairs in three block phases, the chunk's
//     rotations one per lane (a W-th of the rotations' FP64 instructions,
//     at the price of two block barriers per chunk).
// T is the precision of the columns (double; float in the FP32 phase of
// the mixed SVD).
template <typename T, bool CPLX, bool COMP, int STREAM = 0>
__global__ void __launch_bounds__(256, 1) sweeps_kernel(MatViewT<T> M, SvdState *st, double ups,
                                                     int max_sweeps, int rescale_exp, int flags,
                                                     int *lastmod)
{
  __shared__ PairSums s_sums[8];
  __shared__ PairOut s_out[8];
  __shared__ double s_gsum[kGroupWarps];
  if (st->nonfinite) return;
  // STREAM = 1 (four warps per pair, rows in registers) and STREAM = 2 or 4
  // (2 or 4 warps per pair, rows streamed) are instantiations of their own,
  // so that their code and registers bind no other form
  constexpr bool group = STREAM == 1;
  constexpr bool gstream = STREAM >= 2;
  GroupV<CPLX> gv;
  const int nt = M.n + (M.n & 1);
  const int K = nt - 1, L = nt / 2;
  const int lane = threadIdx.x & 31, W = blockDim.x >> 5;
  const bool warp_step = (flags & kFlagWarpStep) != 0;
  // V's transformation held over to the next step (DeferredV) when every
  // warp has at most one pair per step and V's rows take one trip
  const bool defer = !group && !gstream && warp_step && (int64_t)gridDim.x * W >= L &&
                     M.np <= 32 * DeferredV<T, CPLX>::kRows;
  DeferredV<T, CPLX> dv;
  if (K < 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->sweeps = 1;
      st->converged = 1;
    }
    return;
  }
  unsigned long long gstep = 0;
  int sweep = 0;
  bool converged = false;
  int last_rescale = INT_MIN / 2;  // the last step that rescaled G (the same in every block)
  unsigned int bphase = barrier_phase(&st->bar_word);
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int k = 0; k < K; ++k, ++gstep) {
      const int cur = (int)(gstep % 3), nxt = (int)((gstep + 1) % 3), old = (int)((gstep + 2) % 3);
      // a weak L2 load, ordered after the other blocks' updates by the
      // barrier's acquire, which the compiler may issue beside the step's
      // column loads
      const double Mcur = dbl(__ldcg(&st->Mbuf[cur]));
      // section 3.2, step 2: rescale when M~ has grown past 2^rescale_exp
      const int rk =
          (bits(Mcur) != 0ull && flg(Mcur) >= rescale_exp) ? scale_target(rescale_exp) - flg(Mcur) : 0;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->Mbuf[old] = 0ull;
        atomicMax(&st->Mbuf[nxt], bits(rk ? ldexp_rn(Mcur, rk) : Mcur));
        if (rk) {
          st->s += rk;
          st->rescales += 1;
        }
      }
      unsigned long long Mloc = 0ull;
      int rots = 0, gsn = 0;
      if (rk) last_rescale = (int)gstep;
      if constexpr (gstream && !COMP) {
        step_group_stream<T, CPLX, kAccL2, STREAM>(M, k, nt, ups, rk, (flags & kFlagPermute) != 0,
                                                   Mloc, rots, gsn, s_gsum, lastmod, (int)gstep,
                                                   last_rescale);
      } else if constexpr (group) {
        if constexpr (sizeof(T) == 8 && !COMP)
          step_group<CPLX>(M, k, nt, ups, rk, (flags & kFlagPermute) != 0, Mloc, rots, gsn, gv,
                           s_gsum);
      } else if (warp_step)
        step_warps<T, CPLX, COMP>(M, k, nt, ups, rk, (flags & kFlagPermute) != 0, Mloc, rots, gsn,
                                  defer, dv, lastmod, (int)gstep, last_rescale);
      else
        for (int base = blockIdx.x * W; base < L; base += gridDim.x * W)
          step_chunk<T, CPLX, true, COMP>(M, k, nt, base, W, ups, rk, (flags & kFlagPermute) != 0,
                                          s_sums, s_out, Mloc, rots, gsn);
      Mloc = warp_umax(Mloc);
      if (lane == 0) {
        if (Mloc) atomicMax(&st->Mbuf[nxt], bits(magbits_to_double(Mloc, T(0))));
        if (rots) atomicAdd(&st->T[sweep], rots);
        if (gsn) atomicAdd(&st->gs, (unsigned long long)gsn);
      }
      if (!grid_barrier(&st->bar_word, &st->err, kBarrierLimitNs, bphase)) return;
    }
    converged = (((volatile int *)st->T)[sweep] == 0);
  }
  if (defer && dv.p >= 0) {  // the last step's V
    dv.load(M);
    dv.apply(M);
  }
  if constexpr (group && sizeof(T) == 8 && !COMP) {
    if (gv.p >= 0) {
      gv.load(M, threadIdx.x >> 5);
      gv.apply(M, threadIdx.x >> 5);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->sweeps = sweep;
    st->converged = converged ? 1 : 0;
  }
}

// The sweeps of a small matrix inside one thread-block cluster of R = 2^lgR
// blocks (one per SM): the steps are separated by the cluster's hardware
// barrier (barrier.cluster with release / acquire semantics, which orders
// the blocks' global-memory accesses at cluster scope) instead of a grid
// barrier polling global memory, and the running max-norm M~ and the
// sweep's rotation count live in rank 0's shared memory.  G and V stay in
// the workspace, reached through L2 as in sweeps_kernel, and the per-warp
// step is the one of sweeps_kernel (step_warps): the same operations in
// the same order, so the same bits.  (Holding G and V in the blocks'
// shared memory, reached through the cluster's shared window, measured
// slower on GB300: 256 x 128 15.0 vs 14.4 ms.)
constexpr int kClusterMax = 16;

template <typename T, bool CPLX, bool COMP>
__global__ void __launch_bounds__(256, 1) sweeps_cluster_kernel(MatViewT<T> M, SvdState *st,
                                                             double ups, int max_sweeps,
                                                             int rescale_exp, int flags,
                                                             int *lastmod)
{
  namespace cgr = cooperative_groups;
  cgr::cluster_group cluster = cgr::this_cluster();
  __shared__ unsigned long long s_M[3];  // rank 0's is M~ (triple-buffered by step)
  __shared__ int s_T[3];                 // rank 0's counts a sweep's rotations
  if (st->nonfinite) return;  // the same for every block: none reaches a barrier
  const int rank = (int)cluster.block_rank();
  const int nt = M.n + (M.n & 1);
  const int K = nt - 1, L = nt / 2;
  const int lane = threadIdx.x & 31, W = blockDim.x >> 5;
  if (threadIdx.x < 3) {
    s_M[threadIdx.x] = (threadIdx.x == 0) ? ((volatile unsigned long long *)st->Mbuf)[0] : 0ull;
    s_T[threadIdx.x] = 0;
  }
  unsigned long long *M0 = cluster.map_shared_rank(s_M, 0);
  int *T0 = cluster.map_shared_rank(s_T, 0);
  const bool defer = (int64_t)gridDim.x * W >= L && M.np <= 32 * DeferredV<T, CPLX>::kRows;
  DeferredV<T, CPLX> dv;
  cluster.sync();
  if (K < 1) {
    if (rank == 0 && threadIdx.x == 0) {
      st->sweeps = 1;
      st->converged = 1;
    }
    return;
  }
  unsigned long long gstep = 0;
  int sweep = 0;
  bool converged = false;
  int last_rescale = INT_MIN / 2;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    for (int k = 0; k < K; ++k, ++gstep) {
      const int cur = (int)(gstep % 3), nxt = (int)((gstep + 1) % 3), old = (int)((gstep + 2) % 3);
      const double Mcur = dbl(((volatile unsigned long long *)M0)[cur]);
      // section 3.2, step 2: rescale when M~ has grown past 2^rescale_exp
      const int rk =
          (bits(Mcur) != 0ull && flg(Mcur) >= rescale_exp) ? scale_target(rescale_exp) - flg(Mcur) : 0;
      if (rank == 0 && threadIdx.x == 0) {
        s_M[old] = 0ull;
        atomicMax(&s_M[nxt], bits(rk ? ldexp_rn(Mcur, rk) : Mcur));
        if (k == 0) s_T[(sweep + 1) % 3] = 0;  // read last at the end of sweep - 2
        if (rk) {
          st->s += rk;
          st->rescales += 1;
        }
      }
      unsigned long long Mloc = 0ull;
      int rots = 0, gsn = 0;
      if (rk) last_rescale = (int)gstep;
      step_warps<T, CPLX, COMP>(M, k, nt, ups, rk, (flags & kFlagPermute) != 0, Mloc, rots, gsn,
                                defer, dv, lastmod, (int)gstep, last_rescale);
      Mloc = warp_umax(Mloc);
      if (lane == 0) {
        if (Mloc) atomicMax(M0 + nxt, bits(magbits_to_double(Mloc, T(0))));
        if (rots) {
          atomicAdd(T0 + sweep % 3, rots);
          atomicAdd(&st->T[sweep], rots);
        }
        if (gsn) atomicAdd(&st->gs, (unsigned long long)gsn);
      }
      cluster.sync();
    }
    converged = (((volatile int *)T0)[sweep % 3] == 0);
  }
  if (defer && dv.p >= 0) {  // the last step's V
    dv.load(M);
    dv.apply(M);
  }
  if (rank == 0 && threadIdx.x == 0) {
    st->sweeps = sweep;
    st->converged = converged ? 1 : 0;
  }
  cluster.sync();  // no block leaves while another may still read rank 0's counters
}

// Final column norms as (e, f); a zero column gets e = INT_MIN.
template <bool CPLX>
__global__ void colnorm_kernel(MatView M, int *e_out, double *f_out)
{
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  for (int j = w; j < M.n; j += W) colnorm_warp<CPLX>(M, j, lane, e_out, f_out);
}

// rank_j = #{i : sigma_i > sigma_j, or sigma_i == sigma_j and i < j}
__global__ void rank_kernel(int n, const int *e, const double *f, int *rank, SvdState *st,
                            jsvd_info *info, const SvdState *st32)
{
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    rank[j] = rank_of(n, e, f, j);
  if (info && blockIdx.x == 0 && threadIdx.x == 0) {
    jsvd_info out;
    long long rot = 0;
    for (int s = 0; s < st->sweeps && s < kMaxSweepsCap; ++s) rot += st->T[s];
    int sw32 = 0, err32 = 0;
    if (st32) {
      sw32 = st32->sweeps;
      err32 = st32->err;
      for (int s = 0; s < st32->sweeps && s < kMaxSweepsCap; ++s) rot += st32->T[s];
    }
    out.status = st->nonfinite        ? JSVD_E_NONFINITE
                 : (st->err || err32) ? JSVD_E_TIMEOUT
                 : st->converged      ? 0
                                      : JSVD_NOT_CONVERGED;
    out.sweeps = st->sweeps;
    out.rotations = rot;
    out.rescales = st->rescales;
    out.sweeps_fp32 = sw32;
    out.gs_steps = (int32_t)(st->gs > 0x7fffffffull ? 0x7fffffffull : st->gs);
    out.reserved = 0;
    *info = out;
  }
}

// U(:, rank_j) = G(:, j) 2^{-e_j} / f_j; V(:, rank_j) = V_k(:, j);
// sigma(rank_j) = 2^{e_j - s} f_j (section 4.2.1).
template <bool CPLX>
__global__ void output_kernel(MatView M, const int *e, const double *f, const int *rank,
                              const SvdState *st, double *U, int64_t ldu, double *V, int64_t ldv,
                              double *sigma, double *sigma_e, double *sigma_f)
{
  const int s = st->s;
  const bool bad = st->nonfinite != 0;
  for (int j = blockIdx.y; j < M.n; j += gridDim.y) {
    const int r = rank[j];
    const int ej = e[j];
    const double fj = f[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) output_sigma(r, ej, fj, s, bad, sigma, sigma_e, sigma_f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M.m, M.n);
         i += gridDim.x * blockDim.x)
      output_elem<CPLX>(M, i, j, r, ej, fj, bad, U, ldu, V, ldv);
  }
}

// ---------------------------------------------------------------------------

static int g_svd_skip = 1;  // skip the pairs whose columns did not change (same results)

int svd_skip_on() { return g_svd_skip; }

int svd_set_skip(int v)
{
  if (v != 0 && v != 1) return -2;
  g_svd_skip = v;
  return JSVD_OK;
}

static int g_svd_grid_cap = 0;
static int g_svd_warps = 0;
static int g_svd_step = 0;  // 0: four warps per pair with the rows in registers where that
                            // fits, else per warp in one cluster for steps of at most 64
                            // pairs, else two or four warps per pair with the rows streamed up
                            // to 4 pairs per SM, else per warp; 1: chunked; 2: per warp (grid
                            // barrier); 3: per warp in one cluster where it fits; 4: four
                            // warps per pair, rows in registers, where it fits; 5: two or four
                            // warps per pair, rows streamed

int svd_set_step_mode(int v)
{
  if (v < 0 || v > 5) return -2;
  g_svd_step = v;
  return JSVD_OK;
}

int svd_set_grid(int cap, int warps)
{
  if (cap < 0 || cap > (1 << 20)) return -2;
  if (warps != 0 && warps != 1 && warps != 2 && warps != 4 && warps != 8) return -3;
  g_svd_grid_cap = cap;
  g_svd_warps = warps;
  return JSVD_OK;
}

__global__ void ordering_kernel(int n, int32_t *tab)
{
  const int nt = n + (n & 1), K = nt - 1, L = nt / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < K * L; t += gridDim.x * blockDim.x) {
    int p, q;
    pair_of(t / L, t % L, nt, p, q);
    tab[2 * t] = p;
    tab[2 * t + 1] = q;
  }
}

int svd_check_opts(const jsvd_opts *o, int &S, int &mode, int &rexp, int &flags)
{
  S = 100;
  mode = JSVD_FP64;
  rexp = 480;
  flags = 0;
  if (!o) return 0;
  if (o->permute != 0 && o->permute != 1) return -1;
  if (o->compensated != 0 && o->compensated != 1) return -1;
  flags = (o->permute ? kFlagPermute : 0) | (o->compensated ? kFlagComp : 0);
  if (o->max_sweeps > 0) S = o->max_sweeps;
  if (S > kMaxSweepsCap) return -1;
  if (o->mode != JSVD_FP64 && o->mode != JSVD_MIXED_FP32_FP64) return -1;
  mode = o->mode;
  if (o->rescale_exp != 0) {
    if (o->rescale_exp < 1 || o->rescale_exp > 480) return -1;
    rexp = o->rescale_exp;
  }
  return 0;
}


// ---------------------------------------------------------------------------
// mixed precision: FP32 copies of the iteration matrix, FP64 conversion

// G32 = fl32(2^-target G64) (planes: max-norm back in [1, 2) for the FP32
// range), V32 = I, and the FP32 phase's state.
template <bool CPLX>
__global__ void to_fp32_kernel(MatView M64, MatViewT<float> M32, const SvdState *st64,
                               SvdState *st32, int target)
{
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    st32->nonfinite = st64->nonfinite;
    st32->s = st64->s - target;
    st32->Mbuf[0] = st64->Mbuf[0] ? bits(ldexp_rn(dbl(st64->Mbuf[0]), -target)) : 0ull;
  }
  for (int j = blockIdx.y; j < M64.n; j += gridDim.y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M64.mp, M64.np);
         i += gridDim.x * blockDim.x) {
      if (i < M64.mp) {
        M32.gr[j * M32.ldg + i] = __double2float_rn(ldexp_rn(M64.gr[j * M64.ldg + i], -target));
        if (CPLX)
          M32.gi[j * M32.ldg + i] = __double2float_rn(ldexp_rn(M64.gi[j * M64.ldg + i], -target));
      }
      if (i < M64.np) {
        M32.vr[j * M32.ldv + i] = (i == j) ? 1.0f : 0.0f;
        if (CPLX) M32.vi[j * M32.ldv + i] = 0.0f;
      }
    }
  }
}

// V64 = (double) V32 (exact widening)
template <bool CPLX>
__global__ void v_to_fp64_kernel(MatViewT<float> M32, double *vr, double *vi, int64_t ldv)
{
  for (int j = blockIdx.y; j < M32.n; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M32.np; i += gridDim.x * blockDim.x) {
      vr[j * ldv + i] = (double)M32.vr[j * M32.ldv + i];
      if (CPLX) vi[j * ldv + i] = (double)M32.vi[j * M32.ldv + i];
    }
}

// ---------------------------------------------------------------------------
// host side

size_t svd_fp64_workspace(bool cplx, int64_t m, int64_t n) { return svd_layout(cplx, m, n).total; }

// Extra regions of the mixed SVD after the FP64 layout.
struct MixedLayout {
  SvdLayout L;
  size_t st32, g32r, g32i, v32r, v32i, gtr, gti, br, bi, xr, xi, total;
};

static MixedLayout mixed_layout(bool cplx, int64_t m, int64_t n)
{
  MixedLayout X;
  X.L = svd_layout(cplx, m, n);
  size_t o = X.L.total;
  const size_t g32 = sizeof(float) * (size_t)X.L.ldg * (size_t)n;
  const size_t v32 = sizeof(float) * (size_t)X.L.ldv * (size_t)n;
  const size_t g64 = sizeof(double) * (size_t)X.L.ldg * (size_t)n;
  const size_t v64 = sizeof(double) * (size_t)X.L.ldv * (size_t)n;
  X.st32 = o;
  o = align256(o + sizeof(SvdState));
  X.g32r = o;
  o = align256(o + g32);
  X.g32i = o;
  if (cplx) o = align256(o + g32);
  X.v32r = o;
  o = align256(o + v32);
  X.v32i = o;
  if (cplx) o = align256(o + v32);
  X.gtr = o;
  o = align256(o + g64);
  X.gti = o;
  if (cplx) o = align256(o + g64);
  X.br = o;
  o = align256(o + v64);
  X.bi = o;
  if (cplx) o = align256(o + v64);
  X.xr = o;
  o = align256(o + v64);
  X.xi = o;
  if (cplx) o = align256(o + v64);
  X.total = o;
  return X;
}

size_t svd_mixed_workspace(bool cplx, int64_t m, int64_t n) { return mixed_layout(cplx, m, n).total; }

template <typename T>
static MatViewT<T> view_at(char *work, size_t gr, size_t gi, size_t vr, size_t vi, bool cplx,
                           const SvdLayout &L, int64_t m, int64_t n)
{
  MatViewT<T> M;
  M.gr = reinterpret_cast<T *>(work + gr);
  M.gi = cplx ? reinterpret_cast<T *>(work + gi) : nullptr;
  M.vr = reinterpret_cast<T *>(work + vr);
  M.vi = cplx ? reinterpret_cast<T *>(work + vi) : nullptr;
  M.m = (int)m;
  M.n = (int)n;
  M.mp = L.mp;
  M.np = L.np;
  M.ldg = L.ldg;
  M.ldv = L.ldv;
  return M;
}

// A1: ||A||_max, G_1 = 2^{s_0} A (planes) in M, V_1 = I.
template <bool CPLX>
static int phase_init(const MatView &M, const double *A, int64_t lda, SvdState *state, int rexp,
                      cudaStream_t st)
{
  JSVD_SMS(sms);
  const int64_t m = M.m, n = M.n;
  JSVD_CUDA(cudaMemsetAsync(state, 0, sizeof(SvdState), st));
  const int64_t rows = CPLX ? 2 * m : m;
  const int64_t ld = CPLX ? 2 * lda : lda;
  int64_t blocks = (rows * n + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  maxnorm_kernel<<<(int)blocks, 256, 0, st>>>(A, ld, rows, n, &state->M0);
  JSVD_CHECK_LAUNCH();
  dim3 grid((unsigned)((std::max(M.mp, M.np) + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  init_kernel<CPLX><<<grid, 256, 0, st>>>(A, lda, M, state, scale_target(rexp));
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

// The cluster form (sweeps_cluster_kernel) for a matrix whose steps have at
// most kClusterWarps pairs per block of a kClusterMax-block cluster, if the
// GPU can place such a cluster.  Returns JSVD_OK if it launched, 1 if the
// form does not apply.
constexpr int kClusterWarps = 4;

template <typename T, bool CPLX, bool COMP>
static int launch_sweeps_cluster(const MatViewT<T> &M, SvdState *state, double ups, int S,
                                 int rexp, int flags, int *lastmod, cudaStream_t st)
{
  const int nt = M.n + (M.n & 1);
  const int Lp = nt / 2;
  auto kern = sweeps_cluster_kernel<T, CPLX, COMP>;
  for (int R = kClusterMax; R >= 8; R /= 2) {
    if (R * kClusterWarps < Lp) return 1;
    const int W = std::max(1, (Lp + R - 1) / R);
    if (R > 8) JSVD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R);
    cfg.blockDim = dim3(32 * W);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();  // a size this GPU cannot place: try a smaller cluster
      continue;
    }
    if (clusters < 1) continue;
    MatViewT<T> Mk = M;
    JSVD_CUDA(cudaLaunchKernelEx(&cfg, kern, Mk, state, ups, S, rexp, flags, lastmod));
    return JSVD_OK;
  }
  return 1;
}

// A2-A8: every sweep, in one cooperative (or one cluster) launch.
template <typename T, bool CPLX, bool COMP>
static int launch_sweeps(const MatViewT<T> &M, SvdState *state, double ups, int S, int rexp,
                         int flags, int *lastmod, cudaStream_t st)
{
  // the columns' last changes for skipping unchanged pairs (before any step)
  if (!g_svd_skip) lastmod = nullptr;
  if (lastmod) JSVD_CUDA(cudaMemsetAsync(lastmod, 0xFF, sizeof(int) * (size_t)M.n, st));
  const int nt = M.n + (M.n & 1);
  const int Lp = nt / 2;
  JSVD_SMS(sms);
  // four warps on each pair (step_group) for FP64 sweeps of a matrix whose
  // pairs fit one per SM and whose columns fit one load trip
  if constexpr (sizeof(T) == 8 && !COMP) {
    const bool fits = Lp <= sms && M.mp <= 32 * (CPLX ? 4 : 8) &&
                      M.np <= 32 * kGroupWarps * GroupV<CPLX>::kRows;
    if (fits && ((g_svd_step == 0 && g_svd_grid_cap == 0 && g_svd_warps == 0) || g_svd_step == 4)) {
      auto kern = sweeps_kernel<T, CPLX, COMP, 1>;
      int per_sm = 0;
      JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kGroupWarps, 0));
      if (per_sm < 1) return JSVD_E_UNSUPPORTED;
      const int grid = std::max(1, std::min(Lp, per_sm * sms));
      MatViewT<T> Mk = M;
      SvdState *sk = state;
      int Sk = S, rk = rexp, pk = flags;  // the form is the instantiation's
      double upsk = ups;
      int *lm = nullptr;  // the group form forms every pair (its steps are latency-bound)
      void *args[] = {&Mk, &sk, &upsk, &Sk, &rk, &pk, &lm};
      JSVD_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(32 * kGroupWarps),
                                            args, 0, st));
      return JSVD_OK;
    }
  }
  // the cluster form for short steps that the four-warp form does not take
  // (the FP32 phase of the mixed mode, the compensated sums), unless a
  // launch shape for the grid forms is asked for
  const bool auto_form = g_svd_step == 0 && g_svd_grid_cap == 0 && g_svd_warps == 0;
  if (auto_form || g_svd_step == 3) {
    const int rc = launch_sweeps_cluster<T, CPLX, COMP>(M, state, ups, S, rexp, flags, lastmod, st);
    if (rc != 1) return rc;
  }
  // two or four warps on each pair with the rows streamed
  // (step_group_stream): four when every pair of a step gets a block at
  // once, else two when that holds with two.  The default up to 4 pairs per
  // SM; with more pairs each SM already holds enough one-warp pairs
  if constexpr (!COMP) {
    if ((auto_form && Lp <= 4 * sms) || g_svd_step == 5) {
      auto k4 = sweeps_kernel<T, CPLX, COMP, 4>;
      auto k2 = sweeps_kernel<T, CPLX, COMP, 2>;
      int per4 = 0, per2 = 0;
      JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per4, k4, 128, 0));
      JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, 64, 0));
      const bool four = (int64_t)per4 * sms >= Lp || (int64_t)per2 * sms < Lp;
      const int per_sm = four ? per4 : per2;
      if (per_sm < 1) return JSVD_E_UNSUPPORTED;
      const int grid = std::max(1, std::min(Lp, per_sm * sms));
      MatViewT<T> Mk = M;
      SvdState *sk = state;
      int Sk = S, rk = rexp, pk = flags;  // the form is the instantiation's
      double upsk = ups;
      int *lm = lastmod;
      void *args[] = {&Mk, &sk, &upsk, &Sk, &rk, &pk, &lm};
      JSVD_CUDA(cudaLaunchCooperativeKernel(four ? (const void *)k4 : (const void *)k2, dim3(grid),
                                            dim3(four ? 128 : 64), args, 0, st));
      return JSVD_OK;
    }
  }
  // The step form: each warp alone unless the chunked form is asked for.
  // Measured on GB300 for 256 x 128 to 4096 x 2048, real and complex, FP64
  // and mixed: the per-warp form is 2-15 % faster everywhere (its extra
  // FP64 instructions for unshared rotations cost less than the chunked
  // form's block barriers and its coarser spread of pairs over the SMs).
  const bool warp_step = (g_svd_step != 1);
  // warps per block: per-warp form 2, or 1 for FP64 sweeps with more pairs
  // per step than SMs (measured: real 256 x 128 14.56 vs 14.75 ms with 2;
  // complex 4096 x 2048 15.9 vs 16.4 s with 1); chunked form the most (up
  // to 8) that still leave a chunk of pairs for every SM
  int W = g_svd_warps;
  if (W == 0) {
    if (warp_step) {
      W = (sizeof(T) == 4 || Lp <= sms) ? 2 : 1;
    } else {
      W = 1;
      while (W < 8 && (Lp + 2 * W - 1) / (2 * W) >= sms) W *= 2;
    }
  }
  auto kern = sweeps_kernel<T, CPLX, COMP>;
  int per_sm = 0;
  JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W, 0));
  if (per_sm < 1) return JSVD_E_UNSUPPORTED;
  int grid = std::min((Lp + W - 1) / W, per_sm * sms);
  if (g_svd_grid_cap > 0) grid = std::min(grid, g_svd_grid_cap);
  if (grid < 1) grid = 1;
  MatViewT<T> Mk = M;
  SvdState *sk = state;
  int Sk = S, rk = rexp, pk = flags | (warp_step ? kFlagWarpStep : 0);
  double upsk = ups;
  int *lm = warp_step ? lastmod : nullptr;
  void *args[] = {&Mk, &sk, &upsk, &Sk, &rk, &pk, &lm};
  JSVD_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(32 * W), args, 0, st));
  return JSVD_OK;
}

template <typename T, bool CPLX>
static int phase_sweeps(const MatViewT<T> &M, SvdState *state, double ups, int S, int rexp,
                        int flags, int *lastmod, cudaStream_t st)
{
  if constexpr (sizeof(T) == 8) {
    if (flags & kFlagComp)
      return launch_sweeps<T, CPLX, true>(M, state, ups, S, rexp, flags, lastmod, st);
  }
  return launch_sweeps<T, CPLX, false>(M, state, ups, S, rexp, flags, lastmod, st);
}

// A9: norms, order, U = G 2^{-e_j}/f_j, sigma, V, info.
template <bool CPLX>
static int phase_finish(const MatView &M, int *e, double *f, int *rank, SvdState *state,
                        const SvdState *st32, double *U, int64_t ldu, double *sigma,
                        double *sigma_e, double *sigma_f, double *V, int64_t ldv, jsvd_info *info,
                        cudaStream_t st)
{
  JSVD_SMS(sms);
  const int64_t m = M.m, n = M.n;
  const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sms * 8);
  colnorm_kernel<CPLX><<<blocks, 256, 0, st>>>(M, e, f);
  JSVD_CHECK_LAUNCH();
  rank_kernel<<<(int)((n + 127) / 128), 128, 0, st>>>((int)n, e, f, rank, state, info, st32);
  JSVD_CHECK_LAUNCH();
  dim3 grid((unsigned)((std::max<int64_t>(m, n) + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  output_kernel<CPLX><<<grid, 256, 0, st>>>(M, e, f, rank, state, U, ldu, V, ldv, sigma, sigma_e,
                                            sigma_f);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

// The FP64 SVD (Alg. zvjsvd) with V_1 = I.
template <bool CPLX>
static int svd_fp64_run(int64_t m, int64_t n, const double *A, int64_t lda, double *U, int64_t ldu,
                        double *sigma, double *sigma_e, double *sigma_f, double *V, int64_t ldv,
                        char *work, jsvd_info *info, int S, int rexp, int flags,
                        cudaStream_t st)
{
  const SvdLayout L = svd_layout(CPLX, m, n);
  SvdState *state = reinterpret_cast<SvdState *>(work + L.state);
  const MatView M = view_at<double>(work, L.gr, L.gi, L.vr, L.vi, CPLX, L, m, n);
  JSVD_TRY(phase_init<CPLX>(M, A, lda, state, rexp, st));
  // the rank array serves the sweeps as the columns' last-change steps
  JSVD_TRY(phase_sweeps<double, CPLX>(M, state, ldexp(sqrt((double)m), -53), S, rexp, flags,
                                      reinterpret_cast<int *>(work + L.rank), st));
  return phase_finish<CPLX>(M, reinterpret_cast<int *>(work + L.e),
                            reinterpret_cast<double *>(work + L.f),
                            reinterpret_cast<int *>(work + L.rank), state, nullptr, U, ldu, sigma,
                            sigma_e, sigma_f, V, ldv, info, st);
}

// Exponent of the FP32 phase's convergence threshold 2^kMixedTolExp sqrt(m):
// 16 times the FP32 unit roundoff 2^-24, since the lane partial sums of
// that phase are FP32 and carry noise of order sqrt(m) 2^-24; the FP64
// phase finishes the convergence from there.
constexpr int kMixedTolExp = -20;
constexpr int kNewtonSchulzSteps = 2;

// The mixed SVD: FP32 sweeps accumulate V32; V0 = V32 re-orthogonalised in
// FP64 by Newton-Schulz steps X <- X (3I - X^H X)/2; G = 2^{s_0} A V0 by
// FP64 GEMM; FP64 sweeps from (G, V0); finish as the FP64 SVD.
template <bool CPLX>
static int svd_mixed_run_t(int64_t m, int64_t n, const double *A, int64_t lda, double *U,
                           int64_t ldu, double *sigma, double *sigma_e, double *sigma_f, double *V,
                           int64_t ldv, char *work, jsvd_info *info, int S, int rexp, int flags,
                           cudaStream_t st)
{
  const MixedLayout X = mixed_layout(CPLX, m, n);
  const SvdLayout &L = X.L;
  SvdState *st64 = reinterpret_cast<SvdState *>(work + L.state);
  SvdState *st32 = reinterpret_cast<SvdState *>(work + X.st32);
  const MatView M0 = view_at<double>(work, L.gr, L.gi, L.vr, L.vi, CPLX, L, m, n);
  const MatViewT<float> M32 = view_at<float>(work, X.g32r, X.g32i, X.v32r, X.v32i, CPLX, L, m, n);
  const MatView M64 = view_at<double>(work, X.gtr, X.gti, L.vr, L.vi, CPLX, L, m, n);
  double *Br = reinterpret_cast<double *>(work + X.br), *Bi = reinterpret_cast<double *>(work + X.bi);
  double *Xr = reinterpret_cast<double *>(work + X.xr), *Xi = reinterpret_cast<double *>(work + X.xi);
  if (!CPLX) Bi = Xi = nullptr;

  // A1 on the FP64 planes: M0.g = 2^{s_0} A
  JSVD_TRY(phase_init<CPLX>(M0, A, lda, st64, rexp, st));
  // FP32 phase
  JSVD_CUDA(cudaMemsetAsync(st32, 0, sizeof(SvdState), st));
  dim3 grid((unsigned)((std::max(L.mp, L.np) + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  to_fp32_kernel<CPLX><<<grid, 256, 0, st>>>(M0, M32, st64, st32, scale_target(rexp));
  JSVD_CHECK_LAUNCH();
  const double ups32 = ldexp(sqrt((double)m), kMixedTolExp);
  JSVD_TRY(phase_sweeps<float, CPLX>(M32, st32, ups32, S, 1 << 20, flags,
                                     reinterpret_cast<int *>(work + L.rank), st));
  // V0 = orth(V32) in FP64 (in M64.v = the FP64 layout's V planes)
  dim3 gv((unsigned)((L.np + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  v_to_fp64_kernel<CPLX><<<gv, 256, 0, st>>>(M32, M64.vr, M64.vi, L.ldv);
  JSVD_CHECK_LAUNCH();
  // every product runs over the zero-padded rows too, so the padding rows
  // the sweeps read stay exactly zero
  const int ni = (int)n, npi = L.np, mpi = L.mp;
  for (int it = 0; it < kNewtonSchulzSteps; ++it) {
    double *Vr = M64.vr, *Vi = M64.vi;
    // B = V^H V; X = 1.5 V - 0.5 V B; V = X
    if (CPLX) {
      JSVD_TRY(zgemm3m(true, true, ni, ni, npi, 1.0, Vr, Vi, L.ldv, Vr, Vi, L.ldv, 0.0, Br, Bi,
                       L.ldv, st));
      JSVD_CUDA(cudaMemcpyAsync(Xr, Vr, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
      JSVD_CUDA(cudaMemcpyAsync(Xi, Vi, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
      JSVD_TRY(zgemm3m(false, false, npi, ni, ni, -0.5, Vr, Vi, L.ldv, Br, Bi, L.ldv, 1.5, Xr, Xi,
                       L.ldv, st));
      JSVD_CUDA(cudaMemcpyAsync(Vr, Xr, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
      JSVD_CUDA(cudaMemcpyAsync(Vi, Xi, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
    } else {
      JSVD_TRY(dgemm(true, ni, ni, npi, 1.0, Vr, L.ldv, Vr, L.ldv, 0.0, Br, L.ldv, st));
      JSVD_CUDA(cudaMemcpyAsync(Xr, Vr, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
      JSVD_TRY(dgemm(false, npi, ni, ni, -0.5, Vr, L.ldv, Br, L.ldv, 1.5, Xr, L.ldv, st));
      JSVD_CUDA(cudaMemcpyAsync(Vr, Xr, sizeof(double) * L.ldv * n, cudaMemcpyDeviceToDevice, st));
    }
  }
  // G = 2^{s_0} A V0 (FP64 GEMM on the FP64 tensor path)
  if (CPLX)
    JSVD_TRY(zgemm3m(false, false, mpi, ni, ni, 1.0, M0.gr, M0.gi, L.ldg, M64.vr, M64.vi, L.ldv,
                     0.0, M64.gr, M64.gi, L.ldg, st));
  else
    JSVD_TRY(dgemm(false, mpi, ni, ni, 1.0, M0.gr, L.ldg, M64.vr, L.ldv, 0.0, M64.gr, L.ldg, st));
  // the FP64 phase restarts the step state from the max-norm of the new G
  JSVD_CUDA(cudaMemsetAsync(st64->Mbuf, 0, sizeof(st64->Mbuf), st));
  {
    JSVD_SMS(sms);
    int64_t blocks = ((int64_t)L.mp * n + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    maxnorm_kernel<<<(int)blocks, 256, 0, st>>>(M64.gr, L.ldg, L.mp, n, &st64->Mbuf[0]);
    JSVD_CHECK_LAUNCH();
    if (CPLX) {
      maxnorm_kernel<<<(int)blocks, 256, 0, st>>>(M64.gi, L.ldg, L.mp, n, &st64->Mbuf[0]);
      JSVD_CHECK_LAUNCH();
    }
  }
  JSVD_TRY(phase_sweeps<double, CPLX>(M64, st64, ldexp(sqrt((double)m), -53), S, rexp, flags,
                                      reinterpret_cast<int *>(work + L.rank), st));
  return phase_finish<CPLX>(M64, reinterpret_cast<int *>(work + L.e),
                            reinterpret_cast<double *>(work + L.f),
                            reinterpret_cast<int *>(work + L.rank), st64, st32, U, ldu, sigma,
                            sigma_e, sigma_f, V, ldv, info, st);
}

int svd_mixed_run(bool cplx, int64_t m, int64_t n, const void *A, int64_t lda, void *U,
                  int64_t ldu, double *sigma, double *sigma_e, double *sigma_f, void *V,
                  int64_t ldv, char *work, jsvd_info *info, int S, int rexp, int flags,
                  cudaStream_t st)
{
  if (cplx)
    return svd_mixed_run_t<true>(m, n, (const double *)A, lda, (double *)U, ldu, sigma, sigma_e,
                                 sigma_f, (double *)V, ldv, work, info, S, rexp, flags, st);
  return svd_mixed_run_t<false>(m, n, (const double *)A, lda, (double *)U, ldu, sigma, sigma_e,
                                sigma_f, (double *)V, ldv, work, info, S, rexp, flags, st);
}

}  // namespace jsvd

using namespace jsvd;

extern "C" int jsvd_ordering(int32_t n, int32_t *tab, void *stream)
{
  if (n < 2) return -1;
  if (!tab) return -2;
  const int nt = n + (n & 1);
  const int64_t total = (int64_t)(nt - 1) * (nt / 2);
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
  ordering_kernel<<<blocks, 256, 0, as_stream(stream)>>>(n, tab);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

extern "C" int jsvd_svd_workspace_size(jsvd_field field, const jsvd_opts *opts, int64_t m,
                                       int64_t n, size_t *bytes)
{
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int S, mode, rexp, flags;
  if (svd_check_opts(opts, S, mode, rexp, flags)) return -2;
  if (m < 1 || m > (1 << 28)) return -3;
  if (n < 1 || n > m || n > (1 << 20)) return -4;
  if (!bytes) return -5;
  const bool cplx = field == JSVD_COMPLEX;
  *bytes = (mode == JSVD_MIXED_FP32_FP64) ? svd_mixed_workspace(cplx, m, n)
                                          : svd_fp64_workspace(cplx, m, n);
  return JSVD_OK;
}

extern "C" int jsvd_svd(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                        const void *A, int64_t lda, void *U, int64_t ldu, double *sigma,
                        double *sigma_e, double *sigma_f, void *V, int64_t ldv, void *work,
                        size_t work_bytes, jsvd_info *info, void *stream)
{
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int S, mode, rexp, flags;
  if (svd_check_opts(opts, S, mode, rexp, flags)) return -2;
  if (m < 1 || m > (1 << 28)) return -3;
  if (n < 1 || n > m || n > (1 << 20)) return -4;
  const bool cplx = field == JSVD_COMPLEX;
  const uintptr_t al = cplx ? 15 : 7;
  if (!A || ((uintptr_t)A & al)) return -5;
  if (lda < m) return -6;
  if (!U || ((uintptr_t)U & al)) return -7;
  if (ldu < m) return -8;
  if (!sigma) return -9;
  if (!V || ((uintptr_t)V & al)) return -12;
  if (ldv < n) return -13;
  if (!work || ((uintptr_t)work & 255)) return -14;
  size_t need = 0;
  jsvd_svd_workspace_size(field, opts, m, n, &need);
  if (work_bytes < need) return JSVD_E_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  if (mode == JSVD_MIXED_FP32_FP64)
    return svd_mixed_run(cplx, m, n, A, lda, U, ldu, sigma, sigma_e, sigma_f, V, ldv,
                         (char *)work, info, S, rexp, flags, st);
  if (cplx)
    return svd_fp64_run<true>(m, n, (const double *)A, lda, (double *)U, ldu, sigma, sigma_e,
                              sigma_f, (double *)V, ldv, (char *)work, info, S, rexp, flags, st);
  return svd_fp64_run<false>(m, n, (const double *)A, lda, (double *)U, ldu, sigma, sigma_e,
                             sigma_f, (double *)V, ldv, (char *)work, info, S, rexp, flags, st);
}

// ---------------------------------------------------------------------------
// The single precision SVD (binary32 data): the sweeps of the FP32 phase
// (FP32 columns, lane sums combined in FP64, each pair's rotation from the
// FP64 2x2 EVD), the final norms in FP64 from the FP32 columns, binary32
// outputs.  Convergence: |a21'| < fl(eps sqrt m) with eps = 2^-24, the
// binary32 unit roundoff (Eq. e:tol for single precision).

namespace jsvd {

constexpr int kF32TolExp = -24;

struct F32Layout {
  size_t state, gr, gi, vr, vi, e, f, rank, total;
  int mp, np;
};

static F32Layout f32_layout(bool cplx, int64_t m, int64_t n)
{
  F32Layout L;
  L.mp = (int)((m + 31) / 32 * 32);
  L.np = (int)((n + 31) / 32 * 32);
  size_t o = 0;
  L.state = o;
  o = align256(o + sizeof(SvdState));
  L.gr = o;
  o = align256(o + sizeof(float) * (size_t)L.mp * (size_t)n);
  L.gi = o;
  if (cplx) o = align256(o + sizeof(float) * (size_t)L.mp * (size_t)n);
  L.vr = o;
  o = align256(o + sizeof(float) * (size_t)L.np * (size_t)n);
  L.vi = o;
  if (cplx) o = align256(o + sizeof(float) * (size_t)L.np * (size_t)n);
  L.e = o;
  o = align256(o + sizeof(int) * (size_t)n);
  L.f = o;
  o = align256(o + sizeof(double) * (size_t)n);
  L.rank = o;
  o = align256(o + sizeof(int) * (size_t)n);
  L.total = o;
  return L;
}

// max over binary32 entries of |x| (NaN -> Inf), stored as the bits of the
// same value in binary64 (M0 of the state)
__global__ void maxnorm32_kernel(const float *__restrict__ A, int64_t lda, int64_t rows,
                                 int64_t cols, unsigned long long *out)
{
  unsigned int mx = 0u;
  const int64_t total = rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / rows, i = t - j * rows;
    unsigned int a = __float_as_uint(A[j * lda + i]) & 0x7FFFFFFFu;
    a = (a > 0x7F800000u) ? 0x7F800000u : a;
    mx = (a > mx) ? a : mx;
  }
  unsigned long long m64 = (mx >= 0x7F800000u) ? kInf : bits((double)__uint_as_float(mx));
  m64 = warp_umax(m64);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m64);
}

// G32 = fl32(2^s0 A), V32 = I; s0 brings ||A||_max into [2^40, 2^41): high
// in the binary32 range for the room of tiny entries, low enough that no
// lane's sum of squares (at most 2^19 rows) overflows.
constexpr int kF32Target = 40;

template <bool CPLX>
__global__ void init32_kernel(const float *__restrict__ A, int64_t lda, MatViewT<float> M,
                              SvdState *st)
{
  const unsigned long long m0 = st->M0;
  const bool nonfinite = m0 >= kInf;
  const int s0 = (m0 == 0ull || nonfinite) ? 0 : kF32Target - flg(dbl(m0));
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    st->s = s0;
    st->nonfinite = nonfinite ? 1 : 0;
    st->Mbuf[0] = (m0 == 0ull || nonfinite) ? 0ull : bits(ldexp_rn(dbl(m0), s0));
  }
  for (int j = blockIdx.y; j < M.n; j += gridDim.y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M.mp, M.np);
         i += gridDim.x * blockDim.x) {
      if (i < M.mp) {
        float xr = 0.0f, xi = 0.0f;
        if (i < M.m && !nonfinite) {
          if (CPLX) {
            xr = ldexp_rn(A[2 * (j * lda + i)], s0);
            xi = ldexp_rn(A[2 * (j * lda + i) + 1], s0);
          } else {
            xr = ldexp_rn(A[j * lda + i], s0);
          }
        }
        M.gr[j * M.ldg + i] = xr;
        if (CPLX) M.gi[j * M.ldg + i] = xi;
      }
      if (i < M.np) {
        M.vr[j * M.ldv + i] = (i == j) ? 1.0f : 0.0f;
        if (CPLX) M.vi[j * M.ldv + i] = 0.0f;
      }
    }
  }
}

// Final norms: the squares of binary32 entries are exact in binary64 and
// cannot underflow there; sums in the canonical order.
template <bool CPLX>
__global__ void colnorm32_kernel(MatViewT<float> M, int *e_out, double *f_out)
{
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int W = (gridDim.x * blockDim.x) >> 5;
  for (int j = w; j < M.n; j += W) {
    const float *xr = M.gr + j * M.ldg, *xi = CPLX ? M.gi + j * M.ldg : nullptr;
    double s = 0.0;
    for (int i = lane; i < M.mp; i += 32) {
      const double a = (double)ldg2(xr + i);
      s = __fma_rn(a, a, s);
      if (CPLX) {
        const double b = (double)ldg2(xi + i);
        s = __fma_rn(b, b, s);
      }
    }
    s = warp_sum(s);
    if (lane == 0) {
      if (bits(s) == 0ull) {
        e_out[j] = INT_MIN;
        f_out[j] = 1.0;
      } else {
        const double r = __dsqrt_rn(s);
        e_out[j] = flg(r);
        f_out[j] = ldexp_rn(r, -flg(r));
      }
    }
  }
}

// U(:, r) = fl32(G32(:, j) 2^-e / f) (one rounding: the binary64 quotient
// rounded again to binary32 equals the binary32 quotient), V(:, r) = V32,
// sigma_r = fl32(2^(e - s) f).
template <bool CPLX>
__global__ void output32_kernel(MatViewT<float> M, const int *e, const double *f, const int *rank,
                                const SvdState *st, float *U, int64_t ldu, float *V, int64_t ldv,
                                float *sigma)
{
  const int s = st->s;
  const bool bad = st->nonfinite != 0;
  const float nan = __int_as_float(0x7FC00000);
  for (int j = blockIdx.y; j < M.n; j += gridDim.y) {
    const int r = rank[j], ej = e[j];
    const double fj = f[j];
    const bool zero = (ej == INT_MIN);
    if (blockIdx.x == 0 && threadIdx.x == 0)
      sigma[r] = bad ? nan : zero ? 0.0f : __double2float_rn(ldexp_rn(fj, ej - s));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(M.m, M.n);
         i += gridDim.x * blockDim.x) {
      if (i < M.m) {
        float ur = 0.0f, ui = 0.0f;
        if (bad) {
          ur = ui = nan;
        } else if (!zero) {
          ur = __double2float_rn(__ddiv_rn(ldexp_rn((double)M.gr[j * M.ldg + i], -ej), fj));
          if (CPLX) ui = __double2float_rn(__ddiv_rn(ldexp_rn((double)M.gi[j * M.ldg + i], -ej), fj));
        }
        if (CPLX) {
          U[2 * (r * ldu + i)] = ur;
          U[2 * (r * ldu + i) + 1] = ui;
        } else {
          U[r * ldu + i] = ur;
        }
      }
      if (i < M.n) {
        const float vr = bad ? nan : M.vr[j * M.ldv + i];
        if (CPLX) {
          V[2 * (r * ldv + i)] = vr;
          V[2 * (r * ldv + i) + 1] = bad ? nan : M.vi[j * M.ldv + i];
        } else {
          V[r * ldv + i] = vr;
        }
      }
    }
  }
}

template <bool CPLX>
static int svd_f32_run(int64_t m, int64_t n, const float *A, int64_t lda, float *U, int64_t ldu,
                       float *sigma, float *V, int64_t ldv, char *work, jsvd_info *info, int S,
                       int flags, cudaStream_t st)
{
  const F32Layout L = f32_layout(CPLX, m, n);
  SvdState *state = reinterpret_cast<SvdState *>(work + L.state);
  MatViewT<float> M;
  M.gr = reinterpret_cast<float *>(work + L.gr);
  M.gi = CPLX ? reinterpret_cast<float *>(work + L.gi) : nullptr;
  M.vr = reinterpret_cast<float *>(work + L.vr);
  M.vi = CPLX ? reinterpret_cast<float *>(work + L.vi) : nullptr;
  M.m = (int)m;
  M.n = (int)n;
  M.mp = L.mp;
  M.np = L.np;
  M.ldg = L.mp;
  M.ldv = L.np;
  int *e = reinterpret_cast<int *>(work + L.e);
  double *f = reinterpret_cast<double *>(work + L.f);
  int *rank = reinterpret_cast<int *>(work + L.rank);
  JSVD_SMS(sms);
  JSVD_CUDA(cudaMemsetAsync(state, 0, sizeof(SvdState), st));
  const int64_t rows = CPLX ? 2 * m : m, ld = CPLX ? 2 * lda : lda;
  int64_t blocks = (rows * n + 255) / 256;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  maxnorm32_kernel<<<(int)blocks, 256, 0, st>>>(A, ld, rows, n, &state->M0);
  JSVD_CHECK_LAUNCH();
  dim3 grid((unsigned)((std::max(L.mp, L.np) + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  init32_kernel<CPLX><<<grid, 256, 0, st>>>(A, lda, M, state);
  JSVD_CHECK_LAUNCH();
  JSVD_TRY(phase_sweeps<float, CPLX>(M, state, ldexp(sqrt((double)m), kF32TolExp), S, 1 << 20,
                                     flags & kFlagPermute, rank, st));
  const int nb = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)sms * 8);
  colnorm32_kernel<CPLX><<<nb, 256, 0, st>>>(M, e, f);
  JSVD_CHECK_LAUNCH();
  rank_kernel<<<(int)((n + 127) / 128), 128, 0, st>>>((int)n, e, f, rank, state, info, nullptr);
  JSVD_CHECK_LAUNCH();
  dim3 go((unsigned)((std::max<int64_t>(m, n) + 255) / 256), (unsigned)std::min<int64_t>(n, 65535));
  output32_kernel<CPLX><<<go, 256, 0, st>>>(M, e, f, rank, state, U, ldu, V, ldv, sigma);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

}  // namespace jsvd

extern "C" int jsvd_svd_f32_workspace_size(jsvd_field field, const jsvd_opts *opts, int64_t m,
                                           int64_t n, size_t *bytes)
{
  using namespace jsvd;
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int S, mode, rexp, flags;
  if (svd_check_opts(opts, S, mode, rexp, flags)) return -2;
  if (m < 1 || m > (1 << 28)) return -3;
  if (n < 1 || n > m || n > (1 << 20)) return -4;
  if (!bytes) return -5;
  *bytes = f32_layout(field == JSVD_COMPLEX, m, n).total;
  return JSVD_OK;
}

extern "C" int jsvd_svd_f32(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                            const void *A, int64_t lda, void *U, int64_t ldu, float *sigma,
                            void *V, int64_t ldv, void *work, size_t work_bytes, jsvd_info *info,
                            void *stream)
{
  using namespace jsvd;
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int S, mode, rexp, flags;
  if (svd_check_opts(opts, S, mode, rexp, flags) || (flags & kFlagComp)) return -2;
  if (m < 1 || m > (1 << 28)) return -3;
  if (n < 1 || n > m || n > (1 << 20)) return -4;
  const bool cplx = field == JSVD_COMPLEX;
  const uintptr_t al = cplx ? 7 : 3;
  if (!A || ((uintptr_t)A & al)) return -5;
  if (lda < m) return -6;
  if (!U || ((uintptr_t)U & al)) return -7;
  if (ldu < m) return -8;
  if (!sigma) return -9;
  if (!V || ((uintptr_t)V & al)) return -10;
  if (ldv < n) return -11;
  if (!work || ((uintptr_t)work & 255)) return -12;
  if (work_bytes < f32_layout(cplx, m, n).total) return JSVD_E_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  if (cplx)
    return svd_f32_run<true>(m, n, (const float *)A, lda, (float *)U, ldu, sigma, (float *)V, ldv,
                             (char *)work, info, S, flags, st);
  return svd_f32_run<false>(m, n, (const float *)A, lda, (float *)U, ldu, sigma, (float *)V, ldv,
                            (char *)work, info, S, flags, st);
}

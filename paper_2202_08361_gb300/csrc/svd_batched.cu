// svd_batched.cu -- jsvd_svd_batched: one-sided Jacobi SVDs of many matrices
// of uneven sizes in one persistent launch.
//
// Each block takes whole matrices from an atomic queue ordered longest
// first (by m n^2, the cost of a sweep) and runs every phase of the SVD on
// one matrix: the max-norm and scaling of A, all sweeps (one warp per pivot
// pair, __syncthreads between steps, no grid barrier), the final norms,
// the sort and the output.  G and V live in shared memory when they fit the
// launch's budget, else in the matrix's workspace region (L1 and L2).  The arithmetic is that of jsvd_svd (the same
// pair step, the same max-norm and rescaling sequence, the same
// finalisation functions), so a matrix gives the same bits alone through
// jsvd_svd, in any batch, in any position and with any block shape.
#include <algorithm>
#include <climits>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "jsvd_internal.h"
#include "svd_core.cuh"

namespace jsvd {

struct BatchDesc {
  const double *A;
  double *U, *V, *sigma, *sigma_e, *sigma_f;
  int64_t lda, ldu, ldv;
  int64_t off;  // byte offset of the matrix's region in the workspace
  int m, n, mp, np;
};

struct BatchHdr {
  int next;   // queue position
  int count;
  int fp32;   // reserved
  int err;
};

struct BatchLayout {
  size_t hdr, desc, order, regions, total;
};

__host__ __device__ __forceinline__ size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of one matrix's region: G planes, V planes, e, f, rank
static size_t region_bytes(bool cplx, int64_t m, int64_t n)
{
  const int64_t mp = (m + 31) / 32 * 32, np = (n + 31) / 32 * 32;
  const int pl = cplx ? 2 : 1;
  size_t o = 0;
  o = al256(o + sizeof(double) * (size_t)(mp * n) * pl);
  o = al256(o + sizeof(double) * (size_t)(np * n) * pl);
  o = al256(o + sizeof(int) * (size_t)n);
  o = al256(o + sizeof(double) * (size_t)n);
  o = al256(o + sizeof(int) * (size_t)n);
  return o;
}

static BatchLayout batch_layout(int64_t count)
{
  BatchLayout L;
  size_t o = 0;
  L.hdr = o;
  o = al256(o + sizeof(BatchHdr));
  L.desc = o;
  o = al256(o + sizeof(BatchDesc) * (size_t)count);
  L.order = o;
  o = al256(o + sizeof(int) * (size_t)count);
  L.regions = o;
  L.total = o;
  return L;
}

static int g_batch_warps = 0;  // 0: chosen per prepared batch (batch_auto_warps)
static int g_batch_smem_kib = 0;

int batch_set_warps(int w)
{
  if (w != 0 && w != 1 && w != 2 && w != 4 && w != 8 && w != 16) return -2;
  g_batch_warps = w;
  return JSVD_OK;
}

// Warps per block for a batch.  Two things pull apart: many blocks per SM
// hide the pair rotations' latency across matrices (a long batch wants
// small blocks), while a batch that does not fill the GPU wants more warps
// per matrix (more so the larger n).  The rule weighs the batch's count
// against the GPU's capacity in one-warp blocks and its mean n, weighted by
// the cost of a sweep (m n^2).  Measured on GB300 (the best warps): 10,000
// uneven matrices (n up to 256) 2; 1,250 of them 8; 4096 x (64 x 32) 1.
static int batch_auto_warps(int64_t count, const int64_t *m, const int64_t *n, int capacity1)
{
  double w = 0.0, wn = 0.0;
  for (int64_t i = 0; i < count; ++i) {
    const double c = (double)m[i] * (double)n[i] * (double)n[i];
    w += c;
    wn += c * (double)n[i];
  }
  const double navg = (w > 0.0) ? wn / w : 0.0;
  const double x = (count > 0) ? (double)capacity1 / (double)count * (navg / 64.0) : 1.0;
  int warps = 1;
  while (warps < 8 && x >= 1.5 * warps) warps *= 2;
  return warps;
}

// The automatic choice of each prepared workspace, read by the launch (a
// host-side table, so the launch needs no device read and stays capturable).
static std::mutex g_auto_mu;
static std::unordered_map<const void *, int> g_auto_warps;

static void remember_auto(const void *work, int w)
{
  std::lock_guard<std::mutex> lk(g_auto_mu);
  if (g_auto_warps.size() > 4096) g_auto_warps.clear();
  g_auto_warps[work] = w;
}

static int recall_auto(const void *work)
{
  std::lock_guard<std::mutex> lk(g_auto_mu);
  const auto it = g_auto_warps.find(work);
  return it == g_auto_warps.end() ? 8 : it->second;
}

// Largest dynamic shared memory a block may take beside the kernel's static
// arrays (227 KiB per block on sm_103, minus a margin for them).
constexpr int kBatchSmemMaxKiB = 220;

int batch_set_smem(int kib)
{
  if (kib < 0 || kib > kBatchSmemMaxKiB) return -2;
  g_batch_smem_kib = kib;
  return JSVD_OK;
}

// Bytes of shared memory that keep G and V of one matrix (all planes).
__host__ __device__ __forceinline__ size_t smem_need(bool cplx, int mp, int np, int n)
{
  return sizeof(double) * ((size_t)mp + (size_t)np) * (size_t)n * (cplx ? 2 : 1);
}

// Shared state of a block while it works on one matrix.
struct BatchShared {
  int idx;
  unsigned long long M0;
  unsigned long long M[3];
  int T;
  int s;
  int rescales;
  unsigned long long gs;
  PairSums sums[32];
  PairOut out[32];
};

// Every phase of the SVD of one matrix (descriptor d, view M of its G and
// V, e/f/rank scratch in its region) by the whole block.
template <bool CPLX, bool COMP, bool CG>
__device__ __forceinline__ void batch_one(BatchShared &sh, const BatchDesc &d, int idx,
                                          const MatViewT<double, CG> &M, int *e, double *f,
                                          int *rank, jsvd_info *info, int S, int rexp, int flags)
{
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  // A1: max-norm of A (NaN -> Inf), s_0, G_1 = 2^{s_0} A, V_1 = I
  if (threadIdx.x == 0) {
    sh.M0 = 0ull;
    sh.T = 0;
    sh.rescales = 0;
    sh.gs = 0ull;
  }
  __syncthreads();
  {
    const int64_t rows = CPLX ? 2 * (int64_t)d.m : d.m, ld = CPLX ? 2 * d.lda : d.lda;
    unsigned long long mx = 0ull;
    for (int64_t q = threadIdx.x; q < rows * d.n; q += blockDim.x) {
      const int64_t j = q / rows, i = q - j * rows;
      unsigned long long a = abits(d.A[j * ld + i]);
      a = (a > kInf) ? kInf : a;
      mx = (a > mx) ? a : mx;
    }
    mx = warp_umax(mx);
    if (lane == 0) atomicMax(&sh.M0, mx);
  }
  __syncthreads();
  const unsigned long long m0 = sh.M0;
  const bool bad = m0 >= kInf;
  const int s0 = (m0 == 0ull || bad) ? 0 : scale_target(rexp) - flg(dbl(m0));
  for (int64_t q = threadIdx.x; q < (int64_t)d.mp * d.n; q += blockDim.x) {
    const int j = (int)(q / d.mp), i = (int)(q - (int64_t)j * d.mp);
    double xr = 0.0, xi = 0.0;
    if (i < d.m && !bad) {
      if (CPLX) {
        xr = ldexp_rn(d.A[2 * (j * d.lda + i)], s0);
        xi = ldexp_rn(d.A[2 * (j * d.lda + i) + 1], s0);
      } else {
        xr = ldexp_rn(d.A[j * d.lda + i], s0);
      }
    }
    M.st(M.gr + j * M.ldg + i, xr);
    if (CPLX) M.st(M.gi + j * M.ldg + i, xi);
  }
  for (int64_t q = threadIdx.x; q < (int64_t)d.np * d.n; q += blockDim.x) {
    const int j = (int)(q / d.np), i = (int)(q - (int64_t)j * d.np);
    M.st(M.vr + j * M.ldv + i, (i == j) ? 1.0 : 0.0);
    if (CPLX) M.st(M.vi + j * M.ldv + i, 0.0);
  }
  if (threadIdx.x == 0) {
    sh.s = s0;
    sh.M[0] = (m0 == 0ull || bad) ? 0ull : bits(ldexp_rn(dbl(m0), s0));
    sh.M[1] = sh.M[2] = 0ull;
  }
  __syncthreads();

  // A2-A8: the sweeps (as sweeps_kernel, with a block barrier per step)
  int sweeps = 0;
  bool conv = false;
  long long rot_total = 0;
  if (!bad) {
    const int nt = d.n + (d.n & 1), K = nt - 1, L = nt / 2;
    const double ups = ldexp_rn(__dsqrt_rn((double)d.m), -53);  // Eq. e:tol
    if (K < 1) {
      sweeps = 1;
      conv = true;
    }
    unsigned long long gstep = 0;
    // the rank array holds the columns' last-change steps during the sweeps
    // (pairs unchanged since their last meeting are skipped, as in
    // step_warps)
    int *lastmod = (flags & kFlagSkip) ? rank : nullptr;
    if (lastmod)
      for (int j = threadIdx.x; j < d.n; j += blockDim.x) lastmod[j] = -1;
    __syncthreads();
    int last_rescale = INT_MIN / 2;
    for (int sweep = 0; sweep < S && !conv; ++sweep) {
      for (int k = 0; k < K; ++k, ++gstep) {
        const int cur = (int)(gstep % 3), nxt = (int)((gstep + 1) % 3), old = (int)((gstep + 2) % 3);
        const double Mcur = dbl(sh.M[cur]);
        const int rk =
            (bits(Mcur) != 0ull && flg(Mcur) >= rexp) ? scale_target(rexp) - flg(Mcur) : 0;
        if (threadIdx.x == 0) {
          sh.M[old] = 0ull;
          atomicMax(&sh.M[nxt], bits(rk ? ldexp_rn(Mcur, rk) : Mcur));
          if (rk) {
            sh.s += rk;
            sh.rescales += 1;
          }
        }
        unsigned long long Mloc = 0ull;
        int rots = 0, gsn = 0;
        if (rk) last_rescale = (int)gstep;
        for (int base = 0; base < L; base += 32)
          step_chunk<double, CPLX, CG, COMP>(M, k, nt, base, 32, ups, rk,
                                             (flags & kFlagPermute) != 0, sh.sums, sh.out, Mloc,
                                             rots, gsn, lastmod, (int)gstep, last_rescale);
        Mloc = warp_umax(Mloc);
        if (lane == 0) {
          if (Mloc) atomicMax(&sh.M[nxt], Mloc);
          if (rots) atomicAdd(&sh.T, rots);
          if (gsn) atomicAdd(&sh.gs, (unsigned long long)gsn);
        }
        __syncthreads();
      }
      const int T = sh.T;
      rot_total += T;
      sweeps = sweep + 1;
      conv = (T == 0);
      __syncthreads();
      if (threadIdx.x == 0) sh.T = 0;
      __syncthreads();
    }
  }

  // A9: norms, order, outputs, info
  for (int j = warp; j < d.n; j += W) colnorm_warp<CPLX>(M, j, lane, e, f);
  __syncthreads();
  for (int j = threadIdx.x; j < d.n; j += blockDim.x) rank[j] = rank_of(d.n, e, f, j);
  __syncthreads();
  const int sfin = sh.s;
  const int R = max(d.m, d.n);
  for (int64_t q = threadIdx.x; q < (int64_t)R * d.n; q += blockDim.x) {
    const int j = (int)(q / R), i = (int)(q - (int64_t)j * R);
    const int r = rank[j];
    if (i == 0) output_sigma(r, e[j], f[j], sfin, bad, d.sigma, d.sigma_e, d.sigma_f);
    output_elem<CPLX>(M, i, j, r, e[j], f[j], bad, d.U, d.ldu, d.V, d.ldv);
  }
  if (info && threadIdx.x == 0) {
    jsvd_info out;
    out.status = bad ? JSVD_E_NONFINITE : conv ? 0 : JSVD_NOT_CONVERGED;
    out.sweeps = sweeps;
    out.rotations = rot_total;
    out.rescales = sh.rescales;
    out.sweeps_fp32 = 0;
    out.gs_steps = (int32_t)(sh.gs > 0x7fffffffull ? 0x7fffffffull : sh.gs);
    out.reserved = 0;
    info[idx] = out;
  }
}

// One block per matrix at a time; G and V stay in the matrix's region (all
// accesses through L2, ld/st.cg, which measured faster than L1-cached ones
// here), or, when SMEM and they fit in smem_cap bytes, in shared memory.
template <bool CPLX, bool COMP, bool SMEM>
__global__ void __launch_bounds__(512) batched_kernel(const BatchDesc *__restrict__ desc,
                                                       const int *__restrict__ order,
                                                       BatchHdr *hdr, char *work, jsvd_info *info,
                                                       int S, int rexp, int flags,
                                                       size_t smem_cap)
{
  extern __shared__ __align__(16) double s_dyn[];
  __shared__ BatchShared sh;
  const int count = hdr->count;
  for (;;) {
    if (threadIdx.x == 0) sh.idx = atomicAdd(&hdr->next, 1);
    __syncthreads();
    const int t = sh.idx;
    if (t >= count) break;
    const int idx = order[t];
    const BatchDesc d = desc[idx];
    char *reg = work + d.off;
    const size_t gbytes = sizeof(double) * (size_t)d.mp * d.n;
    const size_t vbytes = sizeof(double) * (size_t)d.np * d.n;
    size_t o = (al256(gbytes) + al256(vbytes)) * (CPLX ? 2 : 1);
    int *e = reinterpret_cast<int *>(reg + o);
    o = al256(o + sizeof(int) * (size_t)d.n);
    double *f = reinterpret_cast<double *>(reg + o);
    o = al256(o + sizeof(double) * (size_t)d.n);
    int *rank = reinterpret_cast<int *>(reg + o);
    bool in_smem = false;
    if constexpr (SMEM) in_smem = smem_need(CPLX, d.mp, d.np, d.n) <= smem_cap;
    if (in_smem) {
      const int64_t g = (int64_t)d.mp * d.n, v = (int64_t)d.np * d.n;
      MatViewT<double, false> M;
      M.gr = s_dyn;
      M.gi = CPLX ? s_dyn + g : nullptr;
      M.vr = s_dyn + (CPLX ? 2 * g : g);
      M.vi = CPLX ? s_dyn + 2 * g + v : nullptr;
      M.m = d.m;
      M.n = d.n;
      M.mp = d.mp;
      M.np = d.np;
      M.ldg = d.mp;
      M.ldv = d.np;
      batch_one<CPLX, COMP, false>(sh, d, idx, M, e, f, rank, info, S, rexp, flags);
    } else {
      MatViewT<double, true> M;
      M.gr = reinterpret_cast<double *>(reg);
      M.gi = CPLX ? reinterpret_cast<double *>(reg + al256(gbytes)) : nullptr;
      const size_t ov = al256(gbytes) * (CPLX ? 2 : 1);
      M.vr = reinterpret_cast<double *>(reg + ov);
      M.vi = CPLX ? reinterpret_cast<double *>(reg + ov + al256(vbytes)) : nullptr;
      M.m = d.m;
      M.n = d.n;
      M.mp = d.mp;
      M.np = d.np;
      M.ldg = d.mp;
      M.ldv = d.np;
      batch_one<CPLX, COMP, true>(sh, d, idx, M, e, f, rank, info, S, rexp, flags);
    }
    __syncthreads();
  }
}

static int batch_check(jsvd_field field, const jsvd_opts *opts, int64_t count, const int64_t *m,
                       const int64_t *n, int &S, int &rexp, int &flags)
{
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int mode;
  if (svd_check_opts(opts, S, mode, rexp, flags) || mode != JSVD_FP64) return -2;
  if (count < 0 || count > (1 << 26)) return -3;
  if (count > 0 && (!m || !n)) return -4;
  for (int64_t i = 0; i < count; ++i)
    if (m[i] < 1 || n[i] < 1 || n[i] > m[i] || m[i] > (1 << 24) || n[i] > (1 << 16)) return -4;
  return JSVD_OK;
}

}  // namespace jsvd

using namespace jsvd;

extern "C" int jsvd_svd_batched_workspace_size(jsvd_field field, const jsvd_opts *opts,
                                               int64_t count, const int64_t *m, const int64_t *n,
                                               size_t *bytes)
{
  int S, rexp, flags;
  const int rc = batch_check(field, opts, count, m, n, S, rexp, flags);
  if (rc) return rc;
  if (!bytes) return -6;
  const BatchLayout L = batch_layout(count);
  size_t total = L.regions;
  for (int64_t i = 0; i < count; ++i) total += region_bytes(field == JSVD_COMPLEX, m[i], n[i]);
  *bytes = total;
  return JSVD_OK;
}

extern "C" int jsvd_svd_batched_prepare(jsvd_field field, const jsvd_opts *opts, int64_t count,
                                        const int64_t *m, const int64_t *n, const void *const *A,
                                        const int64_t *lda, void *const *U, const int64_t *ldu,
                                        double *const *sigma, double *const *sigma_e,
                                        double *const *sigma_f, void *const *V,
                                        const int64_t *ldv, void *work, size_t work_bytes,
                                        void *stream)
{
  int S, rexp, flags;
  const int rc = batch_check(field, opts, count, m, n, S, rexp, flags);
  if (rc) return rc;
  if (count > 0 && (!A || !lda || !U || !ldu || !sigma || !V || !ldv)) return -6;
  if (!work || ((uintptr_t)work & 255)) return -15;
  size_t need = 0;
  jsvd_svd_batched_workspace_size(field, opts, count, m, n, &need);
  if (work_bytes < need) return JSVD_E_WORKSPACE;
  const bool cplx = field == JSVD_COMPLEX;
  const uintptr_t al = cplx ? 15 : 7;
  const BatchLayout L = batch_layout(count);
  std::vector<BatchDesc> desc((size_t)count);
  size_t off = L.regions;
  for (int64_t i = 0; i < count; ++i) {
    if (!A[i] || ((uintptr_t)A[i] & al) || lda[i] < m[i]) return -6;
    if (!U[i] || ((uintptr_t)U[i] & al) || ldu[i] < m[i]) return -8;
    if (!sigma[i]) return -10;
    if (!V[i] || ((uintptr_t)V[i] & al) || ldv[i] < n[i]) return -13;
    BatchDesc &d = desc[(size_t)i];
    d.A = (const double *)A[i];
    d.U = (double *)U[i];
    d.V = (double *)V[i];
    d.sigma = sigma[i];
    d.sigma_e = sigma_e ? sigma_e[i] : nullptr;
    d.sigma_f = sigma_f ? sigma_f[i] : nullptr;
    d.lda = lda[i];
    d.ldu = ldu[i];
    d.ldv = ldv[i];
    d.m = (int)m[i];
    d.n = (int)n[i];
    d.mp = (int)((m[i] + 31) / 32 * 32);
    d.np = (int)((n[i] + 31) / 32 * 32);
    d.off = (int64_t)off;
    off += region_bytes(cplx, m[i], n[i]);
  }
  // queue order: longest first (m n^2 of a sweep), ties by index; only the
  // order in which blocks take matrices depends on it, never a result
  std::vector<int> ord((size_t)count);
  for (int64_t i = 0; i < count; ++i) ord[(size_t)i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    const double ca = (double)m[a] * (double)n[a] * (double)n[a];
    const double cb = (double)m[b] * (double)n[b] * (double)n[b];
    return ca > cb;
  });
  {
    // the capacity of the GPU in one-warp blocks of this field's kernel
    int per_sm = 0;
    auto k1 = (field == JSVD_COMPLEX) ? batched_kernel<true, false, false>
                                      : batched_kernel<false, false, false>;
    JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, 32, 0));
    JSVD_SMS(sms);
    remember_auto(work, batch_auto_warps(count, m, n, per_sm * sms));
  }
  BatchHdr h = {0, (int)count, 0, 0};
  char *w = (char *)work;
  cudaStream_t st = as_stream(stream);
  JSVD_CUDA(cudaMemcpyAsync(w + L.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  if (count > 0) {
    JSVD_CUDA(cudaMemcpyAsync(w + L.desc, desc.data(), sizeof(BatchDesc) * desc.size(),
                              cudaMemcpyHostToDevice, st));
    JSVD_CUDA(cudaMemcpyAsync(w + L.order, ord.data(), sizeof(int) * ord.size(),
                              cudaMemcpyHostToDevice, st));
  }
  // the host buffers are pageable: the copies have been staged when the
  // calls return, but keep this call synchronous w.r.t. them to be safe
  JSVD_CUDA(cudaStreamSynchronize(st));
  return JSVD_OK;
}

extern "C" int jsvd_svd_batched_launch(jsvd_field field, const jsvd_opts *opts, int64_t count,
                                       void *work, jsvd_info *info, void *stream)
{
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  int S, mode, rexp, flags;
  if (svd_check_opts(opts, S, mode, rexp, flags) || mode != JSVD_FP64) return -2;
  if (svd_skip_on()) flags |= kFlagSkip;  // JSVD_TUNE_SVD_SKIP
  if (count < 0 || count > (1 << 26)) return -3;
  if (!work || ((uintptr_t)work & 255)) return -4;
  if (count == 0) return JSVD_OK;
  const BatchLayout L = batch_layout(count);
  char *w = (char *)work;
  cudaStream_t st = as_stream(stream);
  // rewind the queue (graph-capturable: a memset node)
  JSVD_CUDA(cudaMemsetAsync(w + L.hdr, 0, sizeof(int), st));
  const int threads = 32 * (g_batch_warps ? g_batch_warps : recall_auto(work));
  const size_t smem = (size_t)g_batch_smem_kib * 1024;
  int per_sm = 0;
  const bool cplx = (field == JSVD_COMPLEX);
  const bool comp = (flags & kFlagComp) != 0;
  using Kern = void (*)(const BatchDesc *, const int *, BatchHdr *, char *, jsvd_info *, int, int,
                        int, size_t);
  static const Kern kerns[8] = {batched_kernel<false, false, false>, batched_kernel<false, false, true>,
                                batched_kernel<false, true, false>,  batched_kernel<false, true, true>,
                                batched_kernel<true, false, false>,  batched_kernel<true, false, true>,
                                batched_kernel<true, true, false>,   batched_kernel<true, true, true>};
  const int ki = (cplx ? 4 : 0) + (comp ? 2 : 0) + (smem > 0 ? 1 : 0);
  const Kern kern = kerns[ki];
  // opt in to the dynamic shared memory (static + dynamic may pass the
  // 48 KiB default even when the budget alone does not)
  static int attr_set[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  if (smem > 0 && attr_set[ki] != g_batch_smem_kib) {
    JSVD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set[ki] = g_batch_smem_kib;
  }
  JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) return JSVD_E_UNSUPPORTED;
  JSVD_SMS(sms);
  const int grid = (int)std::min<int64_t>(count, (int64_t)per_sm * sms);
  kern<<<grid, threads, smem, st>>>(reinterpret_cast<const BatchDesc *>(w + L.desc),
                                    reinterpret_cast<const int *>(w + L.order),
                                    reinterpret_cast<BatchHdr *>(w + L.hdr), w, info, S, rexp,
                                    flags, smem);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

extern "C" int jsvd_svd_batched(jsvd_field field, const jsvd_opts *opts, int64_t count,
                                const int64_t *m, const int64_t *n, const void *const *A,
                                const int64_t *lda, void *const *U, const int64_t *ldu,
                                double *const *sigma, double *const *sigma_e,
                                double *const *sigma_f, void *const *V, const int64_t *ldv,
                                void *work, size_t work_bytes, jsvd_info *info, void *stream)
{
  const int rc = jsvd_svd_batched_prepare(field, opts, count, m, n, A, lda, U, ldu, sigma, sigma_e,
                                          sigma_f, V, ldv, work, work_bytes, stream);
  if (rc) return rc;
  return jsvd_svd_batched_launch(field, opts, count, work, info, stream);
}

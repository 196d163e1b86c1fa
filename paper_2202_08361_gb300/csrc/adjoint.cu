// adjoint.cu -- the SVD adjoint for a batch of real matrices, and the sign
// gauge it is used with.
//
// For A = U diag(s) V^T (thin, m >= n, distinct s) and the cotangents Ubar,
// sbar, Vbar of U, s, V (Townsend 2016, "Differentiating the singular value
// decomposition"; Ionescu et al. 2015):
//   J = U^T Ubar, K = V^T Vbar (n x n),
//   inner_ij = F_ij (J_ij - J_ji) s_j + s_i F_ij (K_ij - K_ji)  (i != j),
//   inner_ii = sbar_i,  F_ij = 1 / (s_j^2 - s_i^2),
//   W = U inner + (Ubar - U J) diag(1/s),
//   Abar = W V^T.
// One block per matrix; all operands of a matrix are staged in shared
// memory (3 m n + 4 n n doubles), FP64 throughout.
#include <algorithm>

#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {

__global__ void __launch_bounds__(256) adjoint_kernel(int count, int m, int n,
                                                      const double *__restrict__ U,
                                                      const double *__restrict__ s,
                                                      const double *__restrict__ V,
                                                      const double *__restrict__ Ub,
                                                      const double *__restrict__ sb,
                                                      const double *__restrict__ Vb,
                                                      double *__restrict__ Ab)
{
  extern __shared__ double sm[];
  double *u = sm;                  // m x n, column-major
  double *ub = u + m * n;          // m x n
  double *Wm = ub + m * n;         // m x n: W
  double *v = Wm + m * n;          // n x n
  double *J = v + n * n;           // n x n: U^T Ubar
  double *K = J + n * n;           // n x n: V^T Vbar
  double *X = K + n * n;           // n x n: inner
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int b = blockIdx.x; b < count; b += gridDim.x) {
    const double *Ui = U + (int64_t)b * m * n, *Vi = V + (int64_t)b * n * n;
    const double *Ubi = Ub ? Ub + (int64_t)b * m * n : nullptr;
    const double *Vbi = Vb ? Vb + (int64_t)b * n * n : nullptr;
    const double *si = s + (int64_t)b * n;
    for (int t = tid; t < m * n; t += nt) {
      u[t] = Ui[t];
      ub[t] = Ubi ? Ubi[t] : 0.0;
    }
    for (int t = tid; t < n * n; t += nt) v[t] = Vi[t];
    __syncthreads();
    // J = U^T Ubar, K = V^T Vbar
    for (int t = tid; t < n * n; t += nt) {
      const int i = t % n, j = t / n;
      double acc = 0.0;
      for (int r = 0; r < m; ++r) acc = __fma_rn(u[r + i * m], ub[r + j * m], acc);
      J[t] = acc;
      double acc2 = 0.0;
      if (Vbi)
        for (int r = 0; r < n; ++r) acc2 = __fma_rn(v[r + i * n], Vbi[(int64_t)r + j * n], acc2);
      K[t] = acc2;
    }
    __syncthreads();
    // inner
    for (int t = tid; t < n * n; t += nt) {
      const int i = t % n, j = t / n;
      double val;
      if (i == j) {
        val = sb ? sb[(int64_t)b * n + i] : 0.0;
      } else {
        const double F = 1.0 / (si[j] * si[j] - si[i] * si[i]);
        val = F * (J[i + j * n] - J[j + i * n]) * si[j] + si[i] * F * (K[i + j * n] - K[j + i * n]);
      }
      X[t] = val;
    }
    __syncthreads();
    // W = U inner + (Ubar - U J) diag(1/s)
    for (int t = tid; t < m * n; t += nt) {
      const int r = t % m, j = t / m;
      double a = 0.0, uj = 0.0;
      for (int i = 0; i < n; ++i) {
        const double uri = u[r + i * m];
        a = __fma_rn(uri, X[i + j * n], a);
        uj = __fma_rn(uri, J[i + j * n], uj);
      }
      Wm[t] = a + (ub[t] - uj) / si[j];
    }
    __syncthreads();
    // Abar = W V^T
    double *Abi = Ab + (int64_t)b * m * n;
    for (int t = tid; t < m * n; t += nt) {
      const int r = t % m, c = t / m;
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc = __fma_rn(Wm[r + j * m], v[c + j * n], acc);
      Abi[t] = acc;
    }
    __syncthreads();
  }
}

// Flip each (u_j, v_j) so that the largest-magnitude entry of u_j is
// positive (first index on ties).  One warp per column.
__global__ void sign_gauge_kernel(int count, int m, int n, double *U, double *V)
{
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t col = w; col < (int64_t)count * n; col += W) {
    const int64_t b = col / n;
    const int j = (int)(col - b * n);
    double *u = U + b * m * n + (int64_t)j * m;
    double *v = V + b * n * n + (int64_t)j * n;
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int r = lane; r < m; r += 32) {
      const double a = fabs(u[r]);
      if (a > best) {
        best = a;
        bi = r;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const bool flip = (bi < m) && (u[bi] < 0.0);
    __syncwarp();
    if (flip) {
      for (int r = lane; r < m; r += 32) u[r] = -u[r];
      for (int r = lane; r < n; r += 32) v[r] = -v[r];
    }
  }
}

static size_t adjoint_smem(int m, int n) { return sizeof(double) * (3 * (size_t)m * n + 4 * (size_t)n * n); }

}  // namespace jsvd

using namespace jsvd;

extern "C" int jsvd_svd_adjoint_batched(int64_t count, int64_t m, int64_t n, const double *U,
                                        const double *s, const double *V, const double *Ubar,
                                        const double *sbar, const double *Vbar, double *Abar,
                                        void *stream)
{
  if (count < 0 || count > INT32_MAX) return -1;
  if (m < 1 || m > (1 << 16)) return -2;
  if (n < 1 || n > m) return -3;
  if (count == 0) return JSVD_OK;
  if (!U) return -4;
  if (!s) return -5;
  if (!V) return -6;
  if (!Abar) return -10;
  const size_t smem = adjoint_smem((int)m, (int)n);
  if (smem > 200 * 1024) return JSVD_E_UNSUPPORTED;
  JSVD_CUDA(cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  int per_sm = 0;
  JSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel, 256, smem));
  if (per_sm < 1) return JSVD_E_UNSUPPORTED;
  JSVD_SMS(sms);
  const int grid = (int)std::min<int64_t>(count, (int64_t)per_sm * sms);
  adjoint_kernel<<<grid, 256, smem, as_stream(stream)>>>((int)count, (int)m, (int)n, U, s, V, Ubar,
                                                         sbar, Vbar, Abar);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

extern "C" int jsvd_sign_gauge_batched(int64_t count, int64_t m, int64_t n, double *U, double *V,
                                       void *stream)
{
  if (count < 0 || count > INT32_MAX) return -1;
  if (m < 1 || m > INT32_MAX) return -2;
  if (n < 1 || n > m) return -3;
  if (count == 0) return JSVD_OK;
  if (!U) return -4;
  if (!V) return -5;
  const int64_t warps = count * n;
  JSVD_SMS(sms);
  const int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)sms * 16);
  sign_gauge_kernel<<<blocks, 256, 0, as_stream(stream)>>>((int)count, (int)m, (int)n, U, V);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

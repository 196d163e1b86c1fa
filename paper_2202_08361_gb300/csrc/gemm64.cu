// gemm64.cu -- FP64 GEMM on the FP64 tensor path (DMMA, mma.sync m8n8k4
// f64), for the dense products of the mixed-precision SVD: G = A V0 and the
// Newton-Schulz re-orthogonalisation of the FP32-accumulated V.
//
//   C = alpha op(A) B + beta C, column-major, op(A) = A (M x K) or A^T
//
// 64 x 64 block tiles, K staged through shared memory 16 at a time, four
// warps of 32 x 32 (4 x 4 mma tiles each).  Ragged edges are zero-filled
// on load and masked on store.  On GB300 the FP64 tensor path and the FP64
// FMA pipe deliver the same rate (about 1 TFLOP/s), so the tiling only has
// to keep that single pipe busy.
#include <algorithm>

#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {

constexpr int kBM = 64, kBN = 64, kBK = 16;

__device__ __forceinline__ void dmma(double (&d)[2], double a, double b)
{
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

template <bool TA>
__global__ void __launch_bounds__(128) dgemm_kernel(int M, int N, int K, double alpha,
                                                    const double *__restrict__ A, int64_t lda,
                                                    const double *__restrict__ B, int64_t ldb,
                                                    double beta, double *__restrict__ C, int64_t ldc)
{
  __shared__ double As[kBK][kBM + 2];  // As[k][m] = op(A)(m0 + m, k0 + k)
  __shared__ double Bs[kBK][kBN + 2];  // Bs[k][n] = B(k0 + k, n0 + n)
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const int g = lane >> 2, t4 = lane & 3;
  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kBK) {
    for (int t = threadIdx.x; t < kBM * kBK; t += blockDim.x) {
      int mm, kk;
      if (TA) {
        kk = t % kBK;  // A^T(m, k) = A(k, m): contiguous in k
        mm = t / kBK;
      } else {
        mm = t % kBM;  // A(m, k): contiguous in m
        kk = t / kBM;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TA ? A[(int64_t)gm * lda + gk] : A[(int64_t)gk * lda + gm];
      As[kk][mm] = v;
    }
    for (int t = threadIdx.x; t < kBK * kBN; t += blockDim.x) {
      const int kk = t % kBK, nn = t / kBK;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[(int64_t)gn * ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 4) {
      double a[4], b[4];
      // fragments of m8n8k4: A (8 x 4, row): a = A[g][t4]; B (4 x 8, col): b = B[t4][g]
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk + t4][wm + 8 * i + g];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk + t4][wn + 8 * j + g];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  // C/D fragment: rows g, columns 2 t4 + {0, 1}
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int r = m0 + wm + 8 * i + g, c = n0 + wn + 8 * j + 2 * t4 + e;
        if (r < M && c < N) {
          double *p = C + (int64_t)c * ldc + r;
          const double v = __dmul_rn(alpha, acc[i][j][e]);
          *p = (beta == 0.0) ? v : __fma_rn(beta, *p, v);
        }
      }
}

int dgemm(bool transA, int M, int N, int K, double alpha, const double *A, int64_t lda,
          const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t st)
{
  if (M <= 0 || N <= 0) return JSVD_OK;
  const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN));
  if (transA)
    dgemm_kernel<true><<<grid, 128, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else
    dgemm_kernel<false><<<grid, 128, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

// Complex C = alpha op(A) B + beta C on split planes (4 real products);
// op(A) = A or A^H.  Bi/Ai may not be NULL.  C must not alias A or B.
int zgemm_split(bool conjtransA, int M, int N, int K, double alpha, const double *Ar,
                const double *Ai, int64_t lda, const double *Br, const double *Bi, int64_t ldb,
                double beta, double *Cr, double *Ci, int64_t ldc, cudaStream_t st)
{
  int rc;
  // real part: N: Ar Br - Ai Bi;  H: Ar^T Br + Ai^T Bi
  if ((rc = dgemm(conjtransA, M, N, K, alpha, Ar, lda, Br, ldb, beta, Cr, ldc, st))) return rc;
  if ((rc = dgemm(conjtransA, M, N, K, conjtransA ? alpha : -alpha, Ai, lda, Bi, ldb, 1.0, Cr, ldc,
                  st)))
    return rc;
  // imaginary part: N: Ar Bi + Ai Br;  H: Ar^T Bi - Ai^T Br
  if ((rc = dgemm(conjtransA, M, N, K, alpha, Ar, lda, Bi, ldb, beta, Ci, ldc, st))) return rc;
  return dgemm(conjtransA, M, N, K, conjtransA ? -alpha : alpha, Ai, lda, Br, ldb, 1.0, Ci, ldc, st);
}

}  // namespace jsvd

extern "C" int jsvd_dgemm(int transA, int64_t M, int64_t N, int64_t K, double alpha,
                          const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                          double *C, int64_t ldc, void *stream)
{
  if (transA != 0 && transA != 1) return -1;
  if (M < 0 || M > INT32_MAX) return -2;
  if (N < 0 || N > INT32_MAX) return -3;
  if (K < 0 || K > INT32_MAX) return -4;
  if (K > 0 && M > 0 && !A) return -6;
  if (lda < (transA ? std::max<int64_t>(K, 1) : std::max<int64_t>(M, 1))) return -7;
  if (K > 0 && N > 0 && !B) return -8;
  if (ldb < std::max<int64_t>(K, 1)) return -9;
  if (M > 0 && N > 0 && !C) return -11;
  if (ldc < std::max<int64_t>(M, 1)) return -12;
  return jsvd::dgemm(transA != 0, (int)M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc,
                     jsvd::as_stream(stream));
}

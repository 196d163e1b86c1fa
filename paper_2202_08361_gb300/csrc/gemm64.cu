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

// Complex C = alpha op(A) B + beta C on split planes by the 3M form: three
// real products per tile in place of four,
//   T1 = op(Ar) Br,  T2 = op(Ai) Bi,  T3 = op(Ar +- Ai) (Br + Bi),
//   op(A) = A:    Re = T1 - T2,  Im = (T3 - T1) - T2   (sum Ar + Ai)
//   op(A) = A^H:  Re = T1 + T2,  Im = (T3 - T1) + T2   (sum Ar - Ai)
// all three in one block: the sum planes are formed in shared memory from
// the loaded tiles.  Each entry of the imaginary part then carries a
// rounding error of order K eps (|Ar| + |Ai|)(|Br| + |Bi|), within a
// factor of two of the four-product form's column-wise bound, which is
// what the one-sided Jacobi sweeps that start from G = A V0 depend on.
// 64 x 32 block tiles, four warps of 32 x 16 (three sets of 4 x 2 mma
// tiles).  HERM (op(A) = A^H, B = A, M = N, beta = 0): C = alpha A^H A is
// Hermitian, so blocks wholly below the diagonal return at once and the
// others write entry (r, c), r <= c, and its conjugate at (c, r); the
// diagonal's imaginary part is set to zero.
constexpr int kZM = 64, kZN = 32, kZK = 16;

template <bool TA, bool HERM>
__global__ void __launch_bounds__(128)
    zgemm3m_kernel(int M, int N, int K, double alpha, const double *__restrict__ Ar,
                   const double *__restrict__ Ai, int64_t lda, const double *__restrict__ Br,
                   const double *__restrict__ Bi, int64_t ldb, double beta,
                   double *__restrict__ Cr, double *__restrict__ Ci, int64_t ldc)
{
  // [plane][k][m]: re, im, re +- im; rows padded by 4 doubles so the
  // fragment loads of a half-warp fall in distinct banks
  __shared__ double As[3][kZK][kZM + 4];
  __shared__ double Bs[3][kZK][kZN + 4];
  const int m0 = blockIdx.x * kZM, n0 = blockIdx.y * kZN;
  if (HERM && m0 >= n0 + kZN) return;  // every entry of the block has r > c
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 16;
  const int g = lane >> 2, t4 = lane & 3;
  double acc[3][4][2][2];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc[p][i][j][0] = acc[p][i][j][1] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kZK) {
    for (int t = threadIdx.x; t < kZM * kZK; t += blockDim.x) {
      int mm, kk;
      if (TA) {
        kk = t % kZK;  // A^H(m, k) = conj A(k, m): contiguous in k
        mm = t / kZK;
      } else {
        mm = t % kZM;  // A(m, k): contiguous in m
        kk = t / kZM;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      double vr = 0.0, vi = 0.0;
      if (gm < M && gk < K) {
        const int64_t o = TA ? (int64_t)gm * lda + gk : (int64_t)gk * lda + gm;
        vr = Ar[o];
        vi = Ai[o];
      }
      As[0][kk][mm] = vr;
      As[1][kk][mm] = vi;
      As[2][kk][mm] = TA ? __dsub_rn(vr, vi) : __dadd_rn(vr, vi);
    }
    for (int t = threadIdx.x; t < kZK * kZN; t += blockDim.x) {
      const int kk = t % kZK, nn = t / kZK;
      const int gk = k0 + kk, gn = n0 + nn;
      double vr = 0.0, vi = 0.0;
      if (gk < K && gn < N) {
        vr = Br[(int64_t)gn * ldb + gk];
        vi = Bi[(int64_t)gn * ldb + gk];
      }
      Bs[0][kk][nn] = vr;
      Bs[1][kk][nn] = vi;
      Bs[2][kk][nn] = __dadd_rn(vr, vi);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kZK; kk += 4) {
      double a[3][4], b[3][2];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[p][i] = As[p][kk + t4][wm + 8 * i + g];
#pragma unroll
        for (int j = 0; j < 2; ++j) b[p][j] = Bs[p][kk + t4][wn + 8 * j + g];
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) dmma(acc[p][i][j], a[p][i], b[p][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int r = m0 + wm + 8 * i + g, c = n0 + wn + 8 * j + 2 * t4 + e;
        if (r >= M || c >= N) continue;
        const double t1 = acc[0][i][j][e], t2 = acc[1][i][j][e], t3 = acc[2][i][j][e];
        const double re = TA ? __dadd_rn(t1, t2) : __dsub_rn(t1, t2);
        const double d31 = __dsub_rn(t3, t1);
        const double im = TA ? __dadd_rn(d31, t2) : __dsub_rn(d31, t2);
        const double vr = __dmul_rn(alpha, re), vi = __dmul_rn(alpha, im);
        if (HERM) {
          if (r > c) continue;
          Cr[(int64_t)c * ldc + r] = vr;
          Ci[(int64_t)c * ldc + r] = (r == c) ? 0.0 : vi;
          if (r < c) {
            Cr[(int64_t)r * ldc + c] = vr;
            Ci[(int64_t)r * ldc + c] = -vi;
          }
        } else {
          double *pr = Cr + (int64_t)c * ldc + r, *pi = Ci + (int64_t)c * ldc + r;
          *pr = (beta == 0.0) ? vr : __fma_rn(beta, *pr, vr);
          *pi = (beta == 0.0) ? vi : __fma_rn(beta, *pi, vi);
        }
      }
}

int zgemm3m(bool conjtransA, bool herm, int M, int N, int K, double alpha, const double *Ar,
            const double *Ai, int64_t lda, const double *Br, const double *Bi, int64_t ldb,
            double beta, double *Cr, double *Ci, int64_t ldc, cudaStream_t st)
{
  if (M <= 0 || N <= 0) return JSVD_OK;
  if (herm && (!conjtransA || M != N || beta != 0.0 || Br != Ar || Bi != Ai || ldb != lda))
    return JSVD_E_UNSUPPORTED;
  const dim3 grid((unsigned)((M + kZM - 1) / kZM), (unsigned)((N + kZN - 1) / kZN));
  if (herm)
    zgemm3m_kernel<true, true><<<grid, 128, 0, st>>>(M, N, K, alpha, Ar, Ai, lda, Br, Bi, ldb,
                                                     beta, Cr, Ci, ldc);
  else if (conjtransA)
    zgemm3m_kernel<true, false><<<grid, 128, 0, st>>>(M, N, K, alpha, Ar, Ai, lda, Br, Bi, ldb,
                                                      beta, Cr, Ci, ldc);
  else
    zgemm3m_kernel<false, false><<<grid, 128, 0, st>>>(M, N, K, alpha, Ar, Ai, lda, Br, Bi, ldb,
                                                       beta, Cr, Ci, ldc);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
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

extern "C" int jsvd_zgemm(int transA, int herm, int64_t M, int64_t N, int64_t K, double alpha,
                          const double *Ar, const double *Ai, int64_t lda, const double *Br,
                          const double *Bi, int64_t ldb, double beta, double *Cr, double *Ci,
                          int64_t ldc, void *stream)
{
  if (transA != 0 && transA != 1) return -1;
  if (herm != 0 && herm != 1) return -2;
  if (herm && !transA) return -2;
  if (M < 0 || M > INT32_MAX) return -3;
  if (N < 0 || N > INT32_MAX || (herm && N != M)) return -4;
  if (K < 0 || K > INT32_MAX) return -5;
  if (K > 0 && M > 0 && !Ar) return -7;
  if (K > 0 && M > 0 && !Ai) return -8;
  if (lda < (transA ? std::max<int64_t>(K, 1) : std::max<int64_t>(M, 1))) return -9;
  if (K > 0 && N > 0 && !Br) return -10;
  if (K > 0 && N > 0 && !Bi) return -11;
  if (ldb < std::max<int64_t>(K, 1)) return -12;
  if (herm && (Br != Ar || Bi != Ai || ldb != lda)) return -10;
  if (herm && beta != 0.0) return -13;
  if (M > 0 && N > 0 && !Cr) return -14;
  if (M > 0 && N > 0 && !Ci) return -15;
  if (ldc < std::max<int64_t>(M, 1)) return -16;
  return jsvd::zgemm3m(transA != 0, herm != 0, (int)M, (int)N, (int)K, alpha, Ar, Ai, lda, Br, Bi,
                       ldb, beta, Cr, Ci, ldc, jsvd::as_stream(stream));
}

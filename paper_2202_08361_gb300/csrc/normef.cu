// normef.cu -- jsvd_colnorm_ef: the wide-exponent Frobenius norms of the
// columns of a matrix (supplement SM6, Alg. rnF).
//
// The summation order is a function of m alone, never of the launch:
// columns of at most kShortRows rows take 32 lanes (one warp), longer ones
// 1024 (one block), lane t adding rows t, t + L, t + 2L, ... in ascending
// order with the (e, f) fma step; the lanes' sums are combined by the xor
// butterfly inside each warp and, for 1024 lanes, by the same butterfly
// over the 32 warps' sums.
#include "common.cuh"
#include "normef.cuh"

namespace jsvd {

constexpr int64_t kShortRows = 8192;  // up to here one warp per column
constexpr int kAhead = 8;             // rows a lane loads before it adds them

// Lane t of L adds rows t, t + L, ... of column x (m rows) to r, in
// ascending order; the loads of kAhead rows are issued before their fma
// steps, so the memory latency is paid once per kAhead rows and the order
// (and the bits) stay those of the one-row loop.
template <bool CPLX>
__device__ __forceinline__ void ef_rows(const double *x, int64_t m, int64_t t, int64_t L, EF &r)
{
  for (int64_t i0 = t; i0 < m; i0 += kAhead * L) {
    double vr[kAhead], vi[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      const int64_t i = i0 + u * L;
      vr[u] = vi[u] = 0.0;
      if (i < m) {
        vr[u] = CPLX ? x[2 * i] : x[i];
        if (CPLX) vi[u] = x[2 * i + 1];
      }
    }
#pragma unroll
    for (int u = 0; u < kAhead; ++u) {
      if (i0 + u * L < m) {
        ef_fma_step(vr[u], r);
        if (CPLX) ef_fma_step(vi[u], r);
      }
    }
  }
}


// Column j of A (m rows; complex: interleaved, each row adds Re^2 then
// Im^2): ||a_j|| as (e, f), e written as a double (-inf for zero).
template <bool CPLX>
__global__ void __launch_bounds__(256) colnorm_ef_kernel(int64_t m, int64_t n, const double *A,
                                                         int64_t lda, double *e_out, double *f_out)
{
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = w; j < n; j += nw) {
    const double *x = A + (CPLX ? 2 : 1) * j * lda;
    EF r = {kNegInfE, 1.0};
    ef_rows<CPLX>(x, m, lane, 32, r);
    r = ef_sqrt(ef_warp_sum(r));
    if (lane == 0) {
      e_out[j] = (r.e == kNegInfE) ? -__longlong_as_double((long long)kInf) : (double)r.e;
      f_out[j] = r.f;
    }
  }
}

// Columns of more than kShortRows rows: one 1024-thread block per column.
template <bool CPLX>
__global__ void __launch_bounds__(1024) colnorm_ef_long_kernel(int64_t m, int64_t n, const double *A,
                                                               int64_t lda, double *e_out,
                                                               double *f_out)
{
  __shared__ int s_e[32];
  __shared__ double s_f[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const double *x = A + (CPLX ? 2 : 1) * j * lda;
    EF r = {kNegInfE, 1.0};
    ef_rows<CPLX>(x, m, t, 1024, r);
    r = ef_warp_sum(r);
    if (lane == 0) {
      s_e[warp] = r.e;
      s_f[warp] = r.f;
    }
    __syncthreads();
    if (warp == 0) {
      EF q = {s_e[lane], s_f[lane]};
      q = ef_sqrt(ef_warp_sum(q));
      if (lane == 0) {
        e_out[j] = (q.e == kNegInfE) ? -__longlong_as_double((long long)kInf) : (double)q.e;
        f_out[j] = q.f;
      }
    }
    __syncthreads();
  }
}

}  // namespace jsvd

extern "C" int jsvd_colnorm_ef(jsvd_field field, int64_t m, int64_t n, const void *A, int64_t lda,
                               double *e_out, double *f_out, void *stream)
{
  using namespace jsvd;
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (n == 0) return JSVD_OK;
  if (!e_out || !f_out) return -6;
  if (m > 0 && !A) return -4;
  if (lda < (m > 0 ? m : 1)) return -5;
  cudaStream_t st = as_stream(stream);
  JSVD_SMS(sms);
  if (m > kShortRows) {
    const int64_t cap = (int64_t)sms * 2;
    const int grid = (int)(n < cap ? n : cap);
    if (field == JSVD_COMPLEX)
      colnorm_ef_long_kernel<true><<<grid, 1024, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
    else
      colnorm_ef_long_kernel<false><<<grid, 1024, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
    JSVD_CHECK_LAUNCH();
    return JSVD_OK;
  }
  const int64_t need = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)sms * 8;
  const int grid = (int)(need < cap ? need : cap);
  if (field == JSVD_COMPLEX)
    colnorm_ef_kernel<true><<<grid, 256, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
  else
    colnorm_ef_kernel<false><<<grid, 256, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

// normef.cu -- jsvd_colnorm_ef: the wide-exponent Frobenius norms of the
// columns of a matrix (supplement SM6, Alg. rnF), one warp per column.
#include "common.cuh"
#include "normef.cuh"

namespace jsvd {

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
    for (int64_t i = lane; i < m; i += 32) {
      if (CPLX) {
        ef_fma_step(x[2 * i], r);
        ef_fma_step(x[2 * i + 1], r);
      } else {
        ef_fma_step(x[i], r);
      }
    }
    r = ef_sqrt(ef_warp_sum(r));
    if (lane == 0) {
      e_out[j] = (r.e == kNegInfE) ? -__longlong_as_double((long long)kInf) : (double)r.e;
      f_out[j] = r.f;
    }
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
  const int64_t need = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  const int grid = (int)(need < cap ? need : cap);
  cudaStream_t st = as_stream(stream);
  if (field == JSVD_COMPLEX)
    colnorm_ef_kernel<true><<<grid, 256, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
  else
    colnorm_ef_kernel<false><<<grid, 256, 0, st>>>(m, n, (const double *)A, lda, e_out, f_out);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

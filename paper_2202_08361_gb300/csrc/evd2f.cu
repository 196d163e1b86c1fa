// evd2f.cu -- jsvd_evd2x2_batched_f32: the batched 2x2 Hermitian EVD in
// single precision.
//
// Same layout and structure as the FP64 kernel (one thread per matrix over
// structure-of-arrays streams, grid-stride, streaming loads and stores).
// On GB300 the FP32 pipe is wide, so this kernel is bound by HBM: each
// thread keeps kUnroll matrices in flight to cover the memory latency.
#include "common.cuh"
#include "evd2f.cuh"
#include "jsvd_internal.h"

namespace jsvd {

constexpr int kUnroll = 4;

template <bool CPLX, bool FAST>
__global__ void __launch_bounds__(256) evd2f_kernel(jsvd_evd2_streams_f32 p, int64_t n)
{
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n;
       i0 += stride * kUnroll) {
    float a11[kUnroll], a22[kUnroll], ar[kUnroll], ai[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      a11[u] = a22[u] = ar[u] = ai[u] = 0.0f;
      if (i < n) {
        a11[u] = __ldcs(p.a11 + i);
        a22[u] = __ldcs(p.a22 + i);
        ar[u] = __ldcs(p.a21_re + i);
        ai[u] = CPLX ? __ldcs(p.a21_im + i) : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = i0 + u * stride;
      if (i < n) {
        const Rot2f r = CPLX ? csjac2<FAST>(a11[u], a22[u], ar[u], ai[u])
                             : ssjac2<FAST>(a11[u], a22[u], ar[u]);
        __stcs(p.cos_phi + i, r.cphi);
        __stcs(p.ea_tan_re + i, r.etr);
        if (CPLX) __stcs(p.ea_tan_im + i, r.eti);
        if (p.lambda1) __stcs(p.lambda1 + i, ldexpf_rn(r.l1s, -r.zeta));
        if (p.lambda2) __stcs(p.lambda2 + i, ldexpf_rn(r.l2s, -r.zeta));
        if (p.zeta_p) __stcs(p.zeta_p + i, pack_zp_f(r));
      }
    }
  }
}

// Division: 1 = the branch-free division (div_fast), 0 = the IEEE
// intrinsic as it is (default: measured faster on wide-range batches, 0.32
// vs 0.37 ms for 2^24 real matrices and 0.49 vs 0.62 ms complex, although
// some lanes of a warp take its slow path).  Same bits either way.
static int g_evd32_fast = 0;

int evd2f_set_fast(int v)
{
  if (v != 0 && v != 1) return -2;
  g_evd32_fast = v;
  return JSVD_OK;
}

}  // namespace jsvd

extern "C" int jsvd_evd2x2_batched_f32(jsvd_field field, const jsvd_evd2_streams_f32 *s,
                                       int64_t n, void *stream)
{
  using namespace jsvd;
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  if (!s) return -2;
  if (n < 0) return -3;
  if (n == 0) return JSVD_OK;
  const bool cplx = (field == JSVD_COMPLEX);
  if (!s->a11 || !s->a22 || !s->a21_re || !s->cos_phi || !s->ea_tan_re) return -2;
  if (cplx && (!s->a21_im || !s->ea_tan_im)) return -2;
  int block, per_sm;
  evd2_get_launch(block, per_sm);
  const int64_t need = (n + (int64_t)block * kUnroll - 1) / ((int64_t)block * kUnroll);
  const int64_t cap = (int64_t)sm_count() * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  cudaStream_t st = as_stream(stream);
  if (g_evd32_fast) {
    if (cplx)
      evd2f_kernel<true, true><<<grid, block, 0, st>>>(*s, n);
    else
      evd2f_kernel<false, true><<<grid, block, 0, st>>>(*s, n);
  } else {
    if (cplx)
      evd2f_kernel<true, false><<<grid, block, 0, st>>>(*s, n);
    else
      evd2f_kernel<false, false><<<grid, block, 0, st>>>(*s, n);
  }
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

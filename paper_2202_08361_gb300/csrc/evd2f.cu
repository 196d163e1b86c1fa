// evd2f.cu -- jsvd_evd2x2_batched_f32: the batched 2x2 Hermitian EVD in
// single precision.
//
// Same layout and structure as the FP64 kernel (one thread per matrix over
// structure-of-arrays streams, grid-stride, streaming loads and stores);
// each thread keeps kUnroll matrices in flight to cover the memory latency.
// On wide-range data the kernel is bound by instruction issue: the
// exponent work and the divisions whose quotients leave the normal range.
#include "common.cuh"
#include "evd2f.cuh"
#include "jsvd_internal.h"

namespace jsvd {

constexpr int kUnroll = 4;

template <bool CPLX, int DM>
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
        const Rot2f r = CPLX ? csjac2<DM>(a11[u], a22[u], ar[u], ai[u])
                             : ssjac2<DM>(a11[u], a22[u], ar[u]);
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

// Division placements (fdiv's DM: bit k set = site k by the branch-free
// division); all give the same bits.
constexpr int kEvd32Masks[] = {
    0x00,  // 0: the IEEE division everywhere
    0xFF,  // 1: the branch-free division everywhere
    0xE3,  // 2: o/|a|, tan(phi), the three phase quotients
    0xE1,  // 3: o/|a| and the three phase quotients
    0x21,  // 4: o/|a| and am/aM
    0xC1,  // 5: o/|a|, |Re a21'|/|a21'|, Im a21'/|a21'|
    0x01,  // 6: o/|a| only
    0xE0,  // 7: the three phase quotients only
};
constexpr int kEvd32Placements = (int)(sizeof(kEvd32Masks) / sizeof(kEvd32Masks[0]));
// real, complex: the fastest measured on wide-range 2^24 batches (ms per
// launch for placements 0..7 -- real: .265 .307 .231 .253 .253 .253 .253
// .264; complex: .425 .514 .418 .405 .397 .432 .422 .394)
constexpr int kEvd32Default[2] = {2, 7};
static int g_evd32_placement[2] = {kEvd32Default[0], kEvd32Default[1]};

// v = -1 restores the defaults; fields: 0 both, 1 real, 2 complex.
int evd2f_set_fast(int v, int fields)
{
  if (v < -1 || v >= kEvd32Placements) return -2;
  if (fields < 0 || fields > 2) return -3;
  for (int c = 0; c < 2; ++c)
    if (fields == 0 || fields == c + 1) g_evd32_placement[c] = (v < 0) ? kEvd32Default[c] : v;
  return JSVD_OK;
}

template <bool CPLX, int I>
static void launch_f32(int placement, int grid, int block, cudaStream_t st,
                       const jsvd_evd2_streams_f32 &s, int64_t n)
{
  if constexpr (I < kEvd32Placements) {
    if (placement == I) {
      evd2f_kernel<CPLX, kEvd32Masks[I]><<<grid, block, 0, st>>>(s, n);
      return;
    }
    launch_f32<CPLX, I + 1>(placement, grid, block, st, s, n);
  }
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
  JSVD_SMS(sms);
  const int64_t cap = (int64_t)sms * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  cudaStream_t st = as_stream(stream);
  if (cplx)
    launch_f32<true, 0>(g_evd32_placement[1], grid, block, st, *s, n);
  else
    launch_f32<false, 0>(g_evd32_placement[0], grid, block, st, *s, n);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

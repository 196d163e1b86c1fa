// evd2.cu -- jsvd_evd2x2_batched: the batched 2x2 Hermitian EVD.
//
// One thread per matrix over structure-of-arrays streams (section 2.4.1),
// the GPU form the paper sketches in supplement SM10, here as a persistent
// grid-stride kernel sized to the SM count.  Inputs are read once with
// streaming loads, outputs written with streaming stores; each matrix is
// independent, so any grid shape and any sub-range give the same bits.
// The divisions and square roots are split between the FP64 pipe and the
// integer pipe (correctly rounded either way) so that the two narrow pipes
// share the work.
#include "common.cuh"
#include "evd2.cuh"
#include "jsvd_internal.h"

namespace jsvd {

template <bool CPLX, int MASK>
__global__ void __launch_bounds__(256) evd2_kernel(const double *__restrict__ a11p,
                                                   const double *__restrict__ a22p,
                                                   const double *__restrict__ a21rp,
                                                   const double *__restrict__ a21ip,
                                                   double *__restrict__ cphip,
                                                   double *__restrict__ etrp,
                                                   double *__restrict__ etip,
                                                   double *__restrict__ l1p,
                                                   double *__restrict__ l2p,
                                                   int32_t *__restrict__ zpp, int64_t n)
{
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double a11 = __ldcs(a11p + i), a22 = __ldcs(a22p + i), a21r = __ldcs(a21rp + i);
    Rot2 r;
    if (CPLX) {
      r = zsjac2<MASK>(a11, a22, a21r, __ldcs(a21ip + i));
    } else {
      r = dsjac2<MASK>(a11, a22, a21r);
    }
    __stcs(cphip + i, r.cphi);
    __stcs(etrp + i, r.etr);
    if (CPLX) __stcs(etip + i, r.eti);
    if (l1p) __stcs(l1p + i, ldexp_rn(r.l1s, -r.zeta));
    if (l2p) __stcs(l2p + i, ldexp_rn(r.l2s, -r.zeta));
    if (zpp) __stcs(zpp + i, pack_zp(r));
  }
}

static int g_evd_block = 256;
static int g_evd_blocks_per_sm = 8;
static int g_evd_variant = 5;

// Division/square-root placements (bit k: slot k on the integer pipe; see
// evd2.cuh).  All give the same bits.
constexpr int kEvdMasks[] = {
    0x000,                                  // 0: every division and root on the FP64 pipe
    0x7FF,                                  // 1: all on the integer pipe
    0x7FF & ~(1 << 6),                      // 2: lambda2' on the FP64 pipe
    0x7FF & ~((1 << 5) | (1 << 6)),         // 3: lambda1', lambda2' on the FP64 pipe
    0x7FF & ~((1 << 4) | (1 << 5) | (1 << 6)),  // 4: and 1/sec
    0x7FF & ~((1 << 1) | (1 << 3)),         // 5: both square roots on the FP64 pipe
};
constexpr int kEvdVariants = (int)(sizeof(kEvdMasks) / sizeof(kEvdMasks[0]));

int evd2_set_variant(int v)
{
  if (v < 0 || v >= kEvdVariants) return -2;
  g_evd_variant = v;
  return JSVD_OK;
}

template <bool CPLX, int V>
static void launch_v(int grid, int block, cudaStream_t st, const jsvd_evd2_streams *s, int64_t n)
{
  evd2_kernel<CPLX, kEvdMasks[V]><<<grid, block, 0, st>>>(
      s->a11, s->a22, s->a21_re, CPLX ? s->a21_im : nullptr, s->cos_phi, s->ea_tan_re,
      CPLX ? s->ea_tan_im : nullptr, s->lambda1, s->lambda2, s->zeta_p, n);
}

template <bool CPLX>
static void launch_any(int v, int grid, int block, cudaStream_t st, const jsvd_evd2_streams *s,
                       int64_t n)
{
  switch (v) {
    case 0: launch_v<CPLX, 0>(grid, block, st, s, n); break;
    case 1: launch_v<CPLX, 1>(grid, block, st, s, n); break;
    case 2: launch_v<CPLX, 2>(grid, block, st, s, n); break;
    case 3: launch_v<CPLX, 3>(grid, block, st, s, n); break;
    case 4: launch_v<CPLX, 4>(grid, block, st, s, n); break;
    default: launch_v<CPLX, 5>(grid, block, st, s, n); break;
  }
}

int evd2_set_launch(int block, int blocks_per_sm)
{
  if (block != 64 && block != 128 && block != 256) return -2;
  if (blocks_per_sm < 1 || blocks_per_sm > 64) return -3;
  g_evd_block = block;
  g_evd_blocks_per_sm = blocks_per_sm;
  return JSVD_OK;
}

}  // namespace jsvd

extern "C" int jsvd_evd2x2_batched(jsvd_field field, const jsvd_evd2_streams *s, int64_t n,
                                   void *stream)
{
  using namespace jsvd;
  if (field != JSVD_REAL && field != JSVD_COMPLEX) return -1;
  if (!s) return -2;
  if (n < 0) return -3;
  if (n == 0) return JSVD_OK;
  const bool cplx = (field == JSVD_COMPLEX);
  if (!s->a11 || !s->a22 || !s->a21_re || !s->cos_phi || !s->ea_tan_re) return -2;
  if (cplx && (!s->a21_im || !s->ea_tan_im)) return -2;
  const int block = g_evd_block;
  const int64_t need = (n + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * g_evd_blocks_per_sm;
  const int grid = (int)(need < cap ? need : cap);
  cudaStream_t st = as_stream(stream);
  if (cplx)
    launch_any<true>(g_evd_variant, grid, block, st, s, n);
  else
    launch_any<false>(g_evd_variant, grid, block, st, s, n);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

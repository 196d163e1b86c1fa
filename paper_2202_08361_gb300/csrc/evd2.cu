// evd2.cu -- jsvd_evd2x2_batched: the batched 2x2 Hermitian EVD.
//
// One thread per matrix over structure-of-arrays streams (section 2.4.1),
// the GPU form the paper sketches in supplement SM10, here as a persistent
// grid-stride kernel sized to the SM count.  Inputs are read once with
// streaming loads, outputs written with streaming stores; each matrix is
// independent, so any grid shape and any sub-range give the same bits.
// The divisions and square roots are split between the FP64 pipe and the
// integer pipe (correctly rounded either way) so that the two narrow pipes
// share the work.  (Splitting one launch between warps of two placements was
// measured slower than either alone: the two code paths double the kernel's
// instruction footprint, and instruction-fetch stalls grow.)
#include "common.cuh"
#include "evd2.cuh"
#include "jsvd_internal.h"

namespace jsvd {

struct EvdPtrs {
  const double *a11, *a22, *a21r, *a21i;
  double *cphi, *etr, *eti, *l1, *l2;
  int32_t *zp;
};

// Elements i, i + stride, ... below n, with one division placement.
template <bool CPLX, int MASK>
__device__ __forceinline__ void evd2_range(int64_t i, int64_t stride, int64_t n, const EvdPtrs &p)
{
  for (; i < n; i += stride) {
    const double a11 = __ldcs(p.a11 + i), a22 = __ldcs(p.a22 + i), a21r = __ldcs(p.a21r + i);
    Rot2 r;
    if (CPLX) {
      r = zsjac2<MASK>(a11, a22, a21r, __ldcs(p.a21i + i));
    } else {
      r = dsjac2<MASK>(a11, a22, a21r);
    }
    __stcs(p.cphi + i, r.cphi);
    __stcs(p.etr + i, r.etr);
    if (CPLX) __stcs(p.eti + i, r.eti);
    if (p.l1) __stcs(p.l1 + i, ldexp_rn(r.l1s, -r.zeta));
    if (p.l2) __stcs(p.l2 + i, ldexp_rn(r.l2s, -r.zeta));
    if (p.zp) __stcs(p.zp + i, pack_zp(r));
  }
}

// 256-thread blocks, JSVD_EVD_MIN_BLOCKS resident per SM asked of the
// register allocator: 8 (32 registers) measured fastest for the complex
// kernel and within noise of the best for the real one.
#ifndef JSVD_EVD_MIN_BLOCKS
#define JSVD_EVD_MIN_BLOCKS 8
#endif
template <bool CPLX, int MASK>
__global__ void __launch_bounds__(256, JSVD_EVD_MIN_BLOCKS) evd2_kernel(EvdPtrs p, int64_t n)
{
  evd2_range<CPLX, MASK>((int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                         (int64_t)gridDim.x * blockDim.x, n, p);
}

static int g_evd_block = 256;
static int g_evd_blocks_per_sm = 8;

// Division/square-root placements (bit k: slot k on the integer pipe; see
// evd2.cuh).  All give the same bits.
constexpr int kEvdMasks[] = {
    0x000,                                  // 0: every division and root on the FP64 pipe
    0x7FF,                                  // 1: all on the integer pipe
    0x7FF & ~(1 << 6),                      // 2: lambda2' on the FP64 pipe
    0x7FF & ~((1 << 5) | (1 << 6)),         // 3: lambda1', lambda2' on the FP64 pipe
    0x7FF & ~((1 << 4) | (1 << 5) | (1 << 6)),  // 4: and 1/sec
    0x7FF & ~((1 << 1) | (1 << 3)),         // 5: both rotation square roots on the FP64 pipe
    0x7FF & ~(1 << 3),                      // 6: sqrt(sec^2) on the FP64 pipe
    0x7FF & ~(1 << 1),                      // 7: sqrt(tan2^2 + 1) on the FP64 pipe
};
constexpr int kEvdPlacements = (int)(sizeof(kEvdMasks) / sizeof(kEvdMasks[0]));

// Default placement per field (real, complex), the fastest measured on
// 2^24 wide-range matrices: only sqrt(tan2^2 + 1) on the FP64 pipe, every
// other division and square root on the integer pipe (ms per launch for
// placements 0..7 -- real: 3.65 .922 1.26 1.86 1.96 1.10 .915 .896;
// complex: 6.13 1.41 1.65 2.18 2.28 1.44 1.37 1.36).
constexpr int kEvdDefault[2] = {7, 7};
static int g_evd_placement[2] = {kEvdDefault[0], kEvdDefault[1]};

int evd2_set_variant(int v, int fields)
{
  if (fields < 0 || fields > 2) return -3;
  if (v != -1 && (v < 0 || v >= kEvdPlacements)) return -2;
  for (int f = 0; f < 2; ++f)
    if (fields == 0 || fields == f + 1) g_evd_placement[f] = (v == -1) ? kEvdDefault[f] : v;
  return JSVD_OK;
}

template <bool CPLX, int V = 0>
static void launch_any(int v, int grid, int block, cudaStream_t st, const EvdPtrs &p, int64_t n)
{
  if constexpr (V < kEvdPlacements) {
    if (v == V)
      evd2_kernel<CPLX, kEvdMasks[V]><<<grid, block, 0, st>>>(p, n);
    else
      launch_any<CPLX, V + 1>(v, grid, block, st, p, n);
  }
}

void evd2_get_launch(int &block, int &blocks_per_sm)
{
  block = g_evd_block;
  blocks_per_sm = g_evd_blocks_per_sm;
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
  JSVD_SMS(sms);
  const int64_t cap = (int64_t)sms * g_evd_blocks_per_sm;
  const int grid = (int)(need < cap ? need : cap);
  cudaStream_t st = as_stream(stream);
  const EvdPtrs p{s->a11, s->a22, s->a21_re, cplx ? s->a21_im : nullptr, s->cos_phi, s->ea_tan_re,
                  cplx ? s->ea_tan_im : nullptr, s->lambda1, s->lambda2, s->zeta_p};
  if (cplx)
    launch_any<true>(g_evd_placement[1], grid, block, st, p, n);
  else
    launch_any<false>(g_evd_placement[0], grid, block, st, p, n);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

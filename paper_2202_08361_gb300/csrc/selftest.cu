// selftest.cu -- jsvd_selftest_fp64: the integer-pipe binary64 division and
// square root (fp64soft.cuh) against the FP64 pipe's IEEE instructions on
// generated operands, counting mismatching bit patterns.
#include <algorithm>

#include "common.cuh"
#include "fp64bits.cuh"
#include "fp64soft.cuh"
#include "jsvd_internal.h"

namespace jsvd {

__device__ __forceinline__ uint64_t splitmix(uint64_t x)
{
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// a finite double from one of several families (any bit pattern,
// subnormals, moderate, powers of two, short mantissas, extremes)
__device__ __forceinline__ double family(uint64_t r, uint64_t r2)
{
  switch (r & 7) {
    case 0: {
      uint64_t u = r2;
      if (((u >> 52) & 0x7FF) == 0x7FF) u &= ~(1ull << 62);
      return __longlong_as_double((long long)u);
    }
    case 1: return __longlong_as_double((long long)(r2 & 0x800FFFFFFFFFFFFFull));
    case 2: return ldexp_rn(1.0 + (double)(r2 >> 11) * 0x1p-53, (int)((r2 >> 3) % 200) - 100);
    case 3: return __longlong_as_double((long long)((((r2 >> 5) % 2046 + 1) << 52) + (r2 & 3) - 1));
    case 4: return ldexp_rn((double)((r2 % 4096) + 1), (int)((r2 >> 20) % 100) - 50);
    case 5: return ldexp_rn(1.0 + (double)(r2 >> 11) * 0x1p-53, 1000 + (int)((r2 >> 2) % 23));
    case 6: return ldexp_rn(1.0 + (double)(r2 >> 11) * 0x1p-53, -1022 + (int)((r2 >> 2) % 60));
    default: return 1.0 + (double)(r2 >> 11) * 0x1p-53;
  }
}

__global__ void selftest_kernel(int64_t n, uint64_t seed, unsigned long long *bad)
{
  unsigned long long bd = 0, bs = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = seed + 4 * (uint64_t)i;
    const double a = family(splitmix(k), splitmix(k + 1));
    double b = family(splitmix(k + 2), splitmix(k + 3));
    if ((__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFll) == 0) b = 1.0;
    if (__double_as_longlong(__ddiv_rn(a, b)) != __double_as_longlong(soft::div_rn(a, b))) ++bd;
    const double x = dabs(a);
    if (__double_as_longlong(__dsqrt_rn(x)) != __double_as_longlong(soft::sqrt_rn(x))) ++bs;
  }
  if (bd) atomicAdd(&bad[0], bd);
  if (bs) atomicAdd(&bad[1], bs);
}

}  // namespace jsvd

extern "C" int jsvd_selftest_fp64(int64_t n, uint64_t seed, unsigned long long *mismatches,
                                  void *stream)
{
  if (n < 0) return -1;
  if (!mismatches) return -3;
  if (n == 0) return JSVD_OK;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)jsvd::sm_count() * 8);
  jsvd::selftest_kernel<<<blocks, 256, 0, jsvd::as_stream(stream)>>>(n, seed, mismatches);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

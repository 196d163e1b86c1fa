// selftest.cu -- self-tests that run on the device:
//   jsvd_selftest_fp64: the integer-pipe binary64 division and square root
//     (fp64soft.cuh and the select-based forms of fp64sel.cuh) against the
//     FP64 pipe's IEEE instructions on generated operands, counting
//     mismatching bit patterns;
//   jsvd_selftest_fp32div: the branch-free binary32 division of the single
//     precision EVD (evd2f.cuh) against the FP32 pipe's IEEE division;
//   jsvd_selftest_barrier: the bounded grid barrier of the persistent SVD
//     kernel, with one block that never arrives, so the others' wait runs
//     out and they report JSVD_E_TIMEOUT (no fault, no trap);
//   jsvd_probe_fp64_rate: a throughput probe of the FP64 pipe (FMA, IEEE
//     square root, IEEE division), the denominator of the FP64-pipe
//     rooflines the benchmark reports.
#include <algorithm>

#include "common.cuh"
#include "evd2f.cuh"
#include "fp64bits.cuh"
#include "fp64sel.cuh"
#include "fp64soft.cuh"
#include "jsvd_internal.h"
#include "svd_core.cuh"

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
    const long long q = __double_as_longlong(__ddiv_rn(a, b));
    if (q != __double_as_longlong(soft::div_rn(a, b))) ++bd;
    if (q != __double_as_longlong(soft::div_rn_sel(a, b))) ++bd;
    const double x = dabs(a);
    const long long r = __double_as_longlong(__dsqrt_rn(x));
    if (r != __double_as_longlong(soft::sqrt_rn(x))) ++bs;
    if (r != __double_as_longlong(soft::sqrt_rn_sel(x))) ++bs;
  }
  if (bd) atomicAdd(&bad[0], bd);
  if (bs) atomicAdd(&bad[1], bs);
}

// Barrier state of the self-test (a library-owned device array: the test
// needs no allocation; concurrent calls would share it).
struct BarrierTestState {
  unsigned int word;
  int err, arrivals, finished;
};
static __device__ BarrierTestState g_bar_test;

// Every block takes `rounds` grid barriers; block `absent` (if in range)
// returns at once and never arrives.  status[0] = JSVD_E_TIMEOUT when a
// wait gave up, else JSVD_OK; status[1] = the barriers the blocks completed.
__global__ void barrier_test_kernel(int absent, int rounds, unsigned long long limit_ns,
                                    int32_t *status)
{
  BarrierTestState *b = &g_bar_test;
  if ((int)blockIdx.x == absent) return;
  int done = 0;
  unsigned int phase = barrier_phase(&b->word);
  for (int r = 0; r < rounds; ++r) {
    if (!grid_barrier(&b->word, &b->err, limit_ns, phase)) break;
    ++done;
  }
  if (threadIdx.x == 0) {
    atomicAdd(&b->arrivals, done);
    __threadfence();
    const int present = (int)gridDim.x - ((absent >= 0 && absent < (int)gridDim.x) ? 1 : 0);
    if (atomicAdd(&b->finished, 1) == present - 1) {  // the last block out reports
      __threadfence();
      status[0] = ((volatile int *)&b->err)[0] ? JSVD_E_TIMEOUT : JSVD_OK;
      status[1] = atomicAdd(&b->arrivals, 0);
    }
  }
}

__global__ void barrier_test_reset()
{
  g_bar_test.word = 0u;
  g_bar_test.err = 0;
  g_bar_test.arrivals = 0;
  g_bar_test.finished = 0;
}

}  // namespace jsvd

extern "C" int jsvd_selftest_barrier(int blocks, int absent, int rounds, int64_t limit_ns,
                                     int32_t *status, void *stream)
{
  using namespace jsvd;
  JSVD_SMS(sms);
  if (blocks < 1 || blocks > sms) return -1;
  if (rounds < 1 || rounds > 1000) return -3;
  if (limit_ns < 1000000 || limit_ns > 5000000000ll) return -4;  // 1 ms .. 5 s
  if (!status) return -5;
  cudaStream_t st = as_stream(stream);
  barrier_test_reset<<<1, 1, 0, st>>>();
  JSVD_CHECK_LAUNCH();
  int a = absent;
  int rr = rounds;
  unsigned long long lim = (unsigned long long)limit_ns;
  void *args[] = {&a, &rr, &lim, &status};
  JSVD_CUDA(cudaLaunchCooperativeKernel((const void *)barrier_test_kernel, dim3(blocks), dim3(32),
                                        args, 0, st));
  return JSVD_OK;
}

namespace jsvd {

// a finite float from one of several families (any bit pattern, subnormals,
// powers of two, short significands, near the top, near the normal range's
// bottom, zero, near one)
__device__ __forceinline__ float family32(uint64_t r, uint64_t r2)
{
  const uint32_t u = (uint32_t)r2;
  switch (r & 7) {
    case 0: return fval(((u >> 23) & 0xFF) == 0xFF ? (u & ~(1u << 30)) : u);
    case 1: return fval(u & 0x807FFFFFu);
    case 2: return fval((u & 0x80000000u) | ((((u >> 8) % 254u) + 1u) << 23));
    case 3: return ldexpf_rn((float)((u % 4096u) + 1u), (int)((u >> 16) % 265u) - 160);  // < 2^117
    case 4: return fval((u & 0x80000000u) | ((uint32_t)(250u + (u >> 24) % 5u) << 23) | (u & 0x7FFFFFu));
    case 5: return fval((u & 0x80000000u) | ((uint32_t)(1u + (u >> 24) % 6u) << 23) | (u & 0x7FFFFFu));
    case 6: return (u & 1u) ? 0.0f : -0.0f;
    default: return fval(0x3F800000u | (u & 0x7FFFFFu));
  }
}

__global__ void selftest32_kernel(int64_t n, uint64_t seed, unsigned long long *bad)
{
  unsigned long long bd = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = seed + 4 * (uint64_t)i;
    const float a = family32(splitmix(k), splitmix(k + 1));
    const float b = family32(splitmix(k + 2), splitmix(k + 3));
    const float x = __fdiv_rn(a, b), y = div_fast(a, b);
    const bool both_nan = (x != x) && (y != y);
    if (!both_nan && fbits(x) != fbits(y)) ++bd;
  }
  if (bd) atomicAdd(bad, bd);
}

// Throughput probe of the FP64 pipe: every thread runs kChains independent
// chains of `iters` operations of one kind, so the pipe, not latency,
// limits the rate.  kind 0: x = fma(x, a, b) (the DFMA rate); kind 1: the
// IEEE square root __dsqrt_rn of a fresh operand each time; kind 2: the
// IEEE division __ddiv_rn.  The fresh operands of kinds 1 and 2 come from
// integer increments of a bit pattern and the results are folded with
// integer XOR, so that only the operation itself runs on the FP64 pipe.
// One thread writes the folded value to sink[0] (keeps the work alive).
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(256) probe_fp64_kernel(int kind, int64_t iters, double *sink)
{
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t fold = 0;
  if (kind == 0) {
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 1.0 + 1e-9 * (t + c);
    const double a = 0.999999999, b = 1e-9;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = __fma_rn(x[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) fold ^= bits(x[c]);
  } else {
    uint64_t u[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) u[c] = 0x3FF8000000000000ull + 977ull * (t * kProbeChains + c);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) {
        const double r = (kind == 1) ? __dsqrt_rn(dbl(u[c])) : __ddiv_rn(1.25, dbl(u[c]));
        fold ^= bits(r);
        u[c] += 0x10001ull;
      }
    }
  }
  if (t == 0 || fold == 0x123456789ull) sink[0] = dbl(fold & 0x3FFFFFFFFFFFFFFFull);
}

}  // namespace jsvd

extern "C" int jsvd_probe_fp64_rate(int kind, int64_t iters, int blocks, int threads,
                                    double *sink, void *stream)
{
  if (kind < 0 || kind > 2) return -1;
  if (iters < 1) return -2;
  if (blocks < 1) return -3;
  if (threads < 32 || threads > 256 || threads % 32 != 0) return -4;
  if (!sink) return -5;
  jsvd::probe_fp64_kernel<<<blocks, threads, 0, jsvd::as_stream(stream)>>>(kind, iters, sink);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

extern "C" int jsvd_selftest_fp32div(int64_t n, uint64_t seed, unsigned long long *mismatches,
                                     void *stream)
{
  if (n < 0) return -1;
  if (!mismatches) return -3;
  if (n == 0) return JSVD_OK;
  JSVD_SMS(sms);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  jsvd::selftest32_kernel<<<blocks, 256, 0, jsvd::as_stream(stream)>>>(n, seed, mismatches);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

extern "C" int jsvd_selftest_fp64(int64_t n, uint64_t seed, unsigned long long *mismatches,
                                  void *stream)
{
  if (n < 0) return -1;
  if (!mismatches) return -3;
  if (n == 0) return JSVD_OK;
  JSVD_SMS(sms);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
  jsvd::selftest_kernel<<<blocks, 256, 0, jsvd::as_stream(stream)>>>(n, seed, mismatches);
  JSVD_CHECK_LAUNCH();
  return JSVD_OK;
}

// api.cu -- library-wide entry points: version, error strings, tuning knobs.
#include <mutex>

#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {

static thread_local cudaError_t g_last_cuda = cudaSuccess;

int cuda_fail(cudaError_t e)
{
  g_last_cuda = e;
  return JSVD_E_CUDA;
}

int sm_count(int *out)
{
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  JSVD_CUDA(cudaGetDevice(&dev));
  if (dev < 0) return cuda_fail(cudaErrorInvalidDevice);
  if (dev >= 64) {  // beyond the cache: ask every time
    int v = 0;
    JSVD_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (v <= 0) return cuda_fail(cudaErrorInvalidValue);
    *out = v;
    return JSVD_OK;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    int v = 0;
    JSVD_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    if (v <= 0) return cuda_fail(cudaErrorInvalidValue);
    cache[dev] = v;
  }
  *out = cache[dev];
  return JSVD_OK;
}

}  // namespace jsvd

extern "C" int jsvd_version(void) { return 100; }

extern "C" const char *jsvd_strerror(int code)
{
  switch (code) {
    case JSVD_OK: return "success";
    case JSVD_E_CUDA: return "a CUDA runtime call failed";
    case JSVD_E_NONFINITE: return "the input holds a non-finite value";
    case JSVD_E_TIMEOUT: return "a bounded device-side wait gave up";
    case JSVD_E_WORKSPACE: return "the workspace is too small";
    case JSVD_E_UNSUPPORTED: return "unsupported combination of arguments";
    default: return (code < 0 && code > -32) ? "invalid argument" : "unknown code";
  }
}

extern "C" const char *jsvd_last_cuda_error(void)
{
  return cudaGetErrorString(jsvd::g_last_cuda);
}

extern "C" int jsvd_tune_set(int knob, int value, int value2)
{
  switch (knob) {
    case JSVD_TUNE_EVD_LAUNCH: return jsvd::evd2_set_launch(value, value2);
    case JSVD_TUNE_EVD_ARITH: return jsvd::evd2_set_variant(value, value2);
    case JSVD_TUNE_SVD_GRID: return jsvd::svd_set_grid(value, value2);
    case JSVD_TUNE_BATCH_WARPS: return jsvd::batch_set_warps(value);
    case JSVD_TUNE_BATCH_SMEM: return jsvd::batch_set_smem(value);
    case JSVD_TUNE_EVD32_DIV: return jsvd::evd2f_set_fast(value, value2);
    case JSVD_TUNE_EVD_HOST: return jsvd::evd2_set_host_path(value);
    case JSVD_TUNE_SVD_STEP: return jsvd::svd_set_step_mode(value);
    case JSVD_TUNE_SVD_SKIP: return jsvd::svd_set_skip(value);
    default: return -1;
  }
}

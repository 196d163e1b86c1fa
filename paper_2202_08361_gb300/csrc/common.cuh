// common.cuh -- host-side plumbing shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "jsvd.h"

namespace jsvd {

// Number of SMs of the current device (cached per device) in *out:
// JSVD_OK, or JSVD_E_CUDA when the device or its attribute cannot be read.
int sm_count(int *out);

// Map a CUDA error to the ABI code (JSVD_E_CUDA), remembering the text.
int cuda_fail(cudaError_t e);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

#define JSVD_CHECK_LAUNCH()                                   \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return ::jsvd::cuda_fail(e_);      \
  } while (0)

// Return an ABI code from a call that produces one, unless it is JSVD_OK.
#define JSVD_TRY(...)                 \
  do {                                \
    const int rc_ = (__VA_ARGS__);    \
    if (rc_ != JSVD_OK) return rc_;   \
  } while (0)

// Declare `var` and set it to the current device's SM count, or return
// the error.
#define JSVD_SMS(var)  \
  int var = 0;         \
  JSVD_TRY(::jsvd::sm_count(&var))

#define JSVD_CUDA(call)                                       \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::jsvd::cuda_fail(e_);      \
  } while (0)

}  // namespace jsvd

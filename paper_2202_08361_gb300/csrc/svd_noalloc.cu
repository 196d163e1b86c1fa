// svd_noalloc.cu -- jsvd_svd_noalloc: the SVD of jsvd_svd for callers that
// cannot allocate device memory.
//
// Some callers may not allocate device memory while they run: code inside a
// framework whose caching allocator has already reserved the GPU's memory
// (a further cudaMalloc can fail there, or force the framework to give back
// its cache), latency-critical loops where cudaMalloc's implicit device
// synchronisation is not acceptable, and processes that must fix their
// memory footprint at start-up.  For them this entry point takes its scratch
// from one file-scope device array of a fixed size instead of a workspace
// argument.  It calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array is part of the library's device image: every GPU on which the
// library's module is loaded holds it until the process exits.  Host code
// never passes the array's name to a kernel (on the host that name is only
// a stand-in, not a device address); every call asks cudaGetSymbolAddress
// for the array's address in the current device's current context and
// passes that.  The lookup is a host-side query and allocates nothing once
// the module is loaded; doing it on every call (rather than caching it per
// device) keeps the address right after cudaDeviceReset or when the caller
// makes another context current.
#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[JSVD_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current context.
int noalloc_scratch(void **out)
{
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e);
  if (p == nullptr) return cuda_fail(cudaErrorInvalidSymbol);
  *out = p;
  return JSVD_OK;
}

}  // namespace
}  // namespace jsvd

extern "C" int jsvd_svd_noalloc(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                                const void *A, int64_t lda, void *U, int64_t ldu, double *sigma,
                                double *sigma_e, double *sigma_f, void *V, int64_t ldv,
                                jsvd_info *info, void *stream)
{
  size_t need = 0;
  const int rc = jsvd_svd_workspace_size(field, opts, m, n, &need);
  if (rc != JSVD_OK) return rc;  // -1..-4: field, opts, m, n
  if (need > (size_t)JSVD_NOALLOC_SCRATCH_BYTES) return JSVD_E_WORKSPACE;
  void *scratch = nullptr;
  const int rs = jsvd::noalloc_scratch(&scratch);
  if (rs != JSVD_OK) return rs;
  // jsvd_svd clears the state it needs at the start of every call and
  // overwrites the rest of the scratch before reading it.
  return jsvd_svd(field, opts, m, n, A, lda, U, ldu, sigma, sigma_e, sigma_f, V, ldv, scratch,
                  (size_t)JSVD_NOALLOC_SCRATCH_BYTES, info, stream);
}

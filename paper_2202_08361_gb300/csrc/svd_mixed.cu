// svd_mixed.cu -- the mixed FP32 -> FP64 Jacobi SVD (work in progress).
#include "common.cuh"
#include "jsvd_internal.h"

namespace jsvd {

size_t svd_mixed_workspace(bool cplx, int64_t m, int64_t n) { return svd_fp64_workspace(cplx, m, n); }

int svd_mixed_run(bool, int64_t, int64_t, const void *, int64_t, void *, int64_t, double *, double *,
                  double *, void *, int64_t, char *, jsvd_info *, int, int, int, cudaStream_t)
{
  return JSVD_E_UNSUPPORTED;
}

}  // namespace jsvd

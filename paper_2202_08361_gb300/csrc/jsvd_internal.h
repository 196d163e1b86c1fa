// jsvd_internal.h -- declarations shared between the library's .cu files.
#pragma once
#include "jsvd.h"

namespace jsvd {
int evd2_set_launch(int block, int blocks_per_sm);
int evd2_set_variant(int v, int fields);
void evd2_get_launch(int &block, int &blocks_per_sm);
int svd_set_grid(int cap, int warps);
int batch_set_warps(int w);
int batch_set_smem(int kib);
int evd2f_set_fast(int v, int fields);
int evd2_set_host_path(int v);
int svd_set_step_mode(int v);
int svd_set_skip(int v);
}  // namespace jsvd

#include <cuda_runtime.h>
#include <stddef.h>

namespace jsvd {
// Option bits carried from jsvd_opts to the kernels.
constexpr int kFlagPermute = 1;  // the column swap P during the sweeps
constexpr int kFlagComp = 2;     // compensated dot-products (FP64 sweeps)
constexpr int kFlagWarpStep = 4; // each warp runs its pairs alone (sweep kernel)
constexpr int kFlagSkip = 32;     // batched sweeps skip unchanged pairs
int svd_skip_on();
int svd_check_opts(const jsvd_opts *o, int &S, int &mode, int &rexp, int &flags);
size_t svd_fp64_workspace(bool cplx, int64_t m, int64_t n);
size_t svd_mixed_workspace(bool cplx, int64_t m, int64_t n);
int dgemm(bool transA, int M, int N, int K, double alpha, const double *A, int64_t lda,
          const double *B, int64_t ldb, double beta, double *C, int64_t ldc, cudaStream_t st);
int zgemm3m(bool conjtransA, bool herm, int M, int N, int K, double alpha, const double *Ar,
            const double *Ai, int64_t lda, const double *Br, const double *Bi, int64_t ldb,
            double beta, double *Cr, double *Ci, int64_t ldc, cudaStream_t st);
int svd_mixed_run(bool cplx, int64_t m, int64_t n, const void *A, int64_t lda, void *U,
                  int64_t ldu, double *sigma, double *sigma_e, double *sigma_f, void *V,
                  int64_t ldv, char *work, jsvd_info *info, int S, int rexp, int flags,
                  cudaStream_t st);
}  // namespace jsvd

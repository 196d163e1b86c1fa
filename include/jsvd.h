/*
 * jsvd.h -- C ABI of the GB300 (sm_103a) Jacobi SVD library.
 *
 * The library implements the data-parallel hot path of the one-sided
 * Jacobi-type SVD of Novakovic, "Vectorization of a thread-parallel Jacobi
 * singular value decomposition method" (arXiv 2202.08361):
 *   - the batched, branch-free eigendecomposition of Hermitian (symmetric)
 *     matrices of order two (section 2, Listing 1, Alg. z8jac2 / d8jac2);
 *   - the one-sided Jacobi SVD built on it (sections 3 and 4,
 *     Alg. zvjsvd).
 *
 * Conventions for every entry point:
 *   - Pointers to arrays are DEVICE pointers (cudaMalloc'd or
 *     torch-allocated memory on the current device) unless stated otherwise;
 *     structs passed by pointer (jsvd_evd2_streams, jsvd_opts, ...) live in
 *     HOST memory.  The caller owns every buffer; the library never frees or
 *     keeps a pointer after the call returns (the work is queued on
 *     `stream`, so device buffers must stay alive until it completes).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call is asynchronous with respect to the host unless its
 *     comment says otherwise.
 *   - Return value: JSVD_OK (0) on success; -i when argument i (1-based) is
 *     invalid (nothing is launched then); JSVD_E_* codes below otherwise.
 *   - Floating point is IEEE-754 binary64 with round-to-nearest-even and
 *     full subnormal support (no flush-to-zero).  Results are bit-identical
 *     across batch sizes, sub-ranges of a batch and launch configurations.
 */
#ifndef JSVD_H
#define JSVD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JSVD_API __attribute__((visibility("default")))
#else
#define JSVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define JSVD_OK 0
#define JSVD_E_CUDA (-100)      /* a CUDA runtime call failed */
#define JSVD_E_NONFINITE (-101) /* an input holds Inf or NaN (section 3.2) */
#define JSVD_E_TIMEOUT (-102)   /* a bounded device-side wait gave up */
#define JSVD_E_WORKSPACE (-103) /* the workspace is too small */
#define JSVD_E_UNSUPPORTED (-104)

typedef enum { JSVD_REAL = 0, JSVD_COMPLEX = 1 } jsvd_field;

/* Library version as 10000*major + 100*minor + patch; never fails. */
JSVD_API int jsvd_version(void);

/* Static description of a return code (never NULL; any int is accepted). */
JSVD_API const char *jsvd_strerror(int code);

/* Text of the last CUDA error this host thread saw (after JSVD_E_CUDA). */
JSVD_API const char *jsvd_last_cuda_error(void);

/* Launch-shape knobs.  They are arithmetic-neutral: no setting changes a
 * single result bit, only the speed.  Process-wide; returns -2 or -3 for a
 * value out of range, -1 for an unknown knob.
 *   JSVD_TUNE_EVD_LAUNCH: value = threads per block of the 2x2 EVD kernels
 *     (FP64 and FP32; 64, 128 or 256), value2 = resident blocks per SM
 *     (1..64). */
#define JSVD_TUNE_EVD_LAUNCH 1
/*   JSVD_TUNE_SVD_GRID: value = most blocks of the persistent SVD sweep
 *     kernel (0 = as many as the pair chunks of a step, capped by
 *     residency); value2 = warps per block (1, 2, 4 or 8; 0 = 2 in the
 *     per-warp step form, or 1 for FP64 sweeps with more pairs per step than
 *     SMs; chosen from the number of pairs and SMs in the chunked one). */
#define JSVD_TUNE_SVD_GRID 2
/*   JSVD_TUNE_BATCH_WARPS: value = warps per block of the batched SVD
 *     kernel (1, 2, 4, 8 or 16), or 0 (the default): chosen when the batch
 *     is prepared, from its mean n weighted by m n^2 (1 warp for n ~ 32, 8
 *     for n ~ 256). */
#define JSVD_TUNE_BATCH_WARPS 3
/*   JSVD_TUNE_EVD_ARITH: value = which of the 2x2 EVD's divisions and
 *     square roots run on the integer pipe instead of the FP64 pipe (0..7;
 *     -1 = the default, 7 for both fields); value2 =
 *     the fields it applies to (0 both, 1 real, 2 complex).  Both pipes
 *     round correctly: the results are identical. */
#define JSVD_TUNE_EVD_ARITH 4
/*   JSVD_TUNE_BATCH_SMEM: value = KiB of shared memory per block of the
 *     batched SVD kernel (0..220; default 0).  A matrix whose G and V
 *     (padded rows, all planes) fit in it is iterated there instead of in
 *     its workspace region. */
#define JSVD_TUNE_BATCH_SMEM 5
/*   JSVD_TUNE_EVD32_DIV: which divisions of the single precision EVD use a
 *     branch-free routine (operands scaled into [1, 2), the quotient's
 *     exponent rebuilt, subnormal results rounded with the exact remainder)
 *     instead of the IEEE division: value = a placement 0..7 (0 none, 1 all,
 *     2 o/|a|, tan(phi) and the phase quotients of a21', 3 - 7 subsets of
 *     these; -1 = the defaults, 2 for real and 7 -- the phase quotients only --
 *     for complex matrices); value2 = the fields it
 *     applies to (0 both, 1 real, 2 complex).  All round correctly: the
 *     results are identical. */
#define JSVD_TUNE_EVD32_DIV 6
/*   JSVD_TUNE_EVD_HOST: how jsvd_evd2x2_batched_host moves its data.
 *     value = 0 (default): directly, the kernel reading and writing the host
 *     streams, when every stream is page-locked memory mapped for the
 *     current device, else staged; 1: always staged through the workspace
 *     in chunks.  The results are identical. */
#define JSVD_TUNE_EVD_HOST 7
/*   JSVD_TUNE_SVD_STEP: the form of a step in the single-matrix sweep
 *     kernel: 0 (the default) = four warps on each pair, the rows in
 *     registers, where a step's pairs fit one per SM and the columns one
 *     load trip; else each warp alone in one thread-block cluster for steps
 *     of at most 64 pairs; else two or four warps on each pair with the rows
 *     streamed, up to 4 pairs per SM; else each warp alone.  1 = chunks of
 *     pairs in three block phases, one pair's rotation per lane; 2 = each
 *     warp runs its pairs alone, a rotation's independent divisions and
 *     square roots spread over its lanes, steps separated by a grid barrier;
 *     3 = the same in one cluster where it fits; 4 = four warps per pair,
 *     rows in registers, where it fits; 5 = two or four warps per pair, rows
 *     streamed.  The results are identical. */
#define JSVD_TUNE_SVD_STEP 8
/*   JSVD_TUNE_SVD_SKIP: value = 1 (default): the sweeps (single-matrix and
 *     batched) skip a pivot pair neither of whose columns has changed since
 *     the pair was last taken, one sweep earlier (its rotation test would
 *     fail again on the same columns); 0: every pair is formed.  A batched
 *     launch takes the value in force when it is launched (or captured).
 *     The results are identical. */
#define JSVD_TUNE_SVD_SKIP 9
/* Sets one of the knobs above for the whole process (not thread-safe with
 * respect to launches running concurrently on other host threads).
 * Errors: -1 unknown knob, -2 value out of range, -3 value2 out of range. */
JSVD_API int jsvd_tune_set(int knob, int value, int value2);

/* ------------------------------------------------------------------------
 * Batched eigendecomposition of Hermitian matrices of order two.
 *
 * Defined by section 2 of the paper: Listing 1 (zsjac2) for the complex
 * case, Alg. d8jac2 (supplement SM2.1) for the real one: the branch-free
 * rotation of section 2.1 (Eq. e:jaclam to e:lamsec), the power-of-two
 * prescaling of Eq. e:z that keeps every output finite (Prop. p:s2), in
 * the structure-of-arrays layout of section 2.4.1 (Eq. e:layout1), with
 * the packed exponent/permutation word of supplement SM10.  Each matrix
 *     A = [ a11        conj(a21) ]
 *         [ a21        a22       ]
 * is factored as A = U Lambda U^*, with
 *     U = cos(phi) [ 1                   -conj(e^{i alpha} tan(phi)) ]
 *                  [ e^{i alpha} tan(phi) 1                          ].
 *
 * Streams (all length n, double unless stated, contiguous, no alignment
 * or padding requirement; output streams must not alias input streams):
 *   in : a11, a22, a21_re, a21_im (a21_im is ignored for JSVD_REAL and may
 *        be NULL there).  All entries must be finite.
 *   out: cos_phi    cos(phi) in [fl(1/sqrt 2), 1]
 *        ea_tan_re  REAL: sign(a21) tan(phi); COMPLEX: cos(alpha) tan(phi)
 *        ea_tan_im  COMPLEX: sin(alpha) tan(phi) (unused for REAL, may be
 *                   NULL there)
 *        lambda1, lambda2   eigenvalues 2^{-zeta} lambda', backscaled with a
 *                   single rounding (may overflow to +-Inf or lose low bits
 *                   as subnormals when the input spans the whole range;
 *                   lambda' itself is always finite); may be NULL
 *        zeta_p     int32 (zeta' << 1) | p, zeta' = -zeta (Eq. e:z, in
 *                   [-2094, 3]), p = 1 iff lambda1' < lambda2' (the column
 *                   swap of section 2); may be NULL.
 * n = 0 is a no-op (the stream pointers are not looked at).  Errors: -1 bad
 * field, -2 NULL streams or a required stream pointer NULL, -3 n < 0,
 * JSVD_E_CUDA on a launch failure.
 */
typedef struct {
  const double *a11, *a22, *a21_re, *a21_im;
  double *cos_phi, *ea_tan_re, *ea_tan_im;
  double *lambda1, *lambda2;
  int32_t *zeta_p;
} jsvd_evd2_streams;

JSVD_API int jsvd_evd2x2_batched(jsvd_field field, const jsvd_evd2_streams *s, int64_t n, void *stream);

/* The same batched EVD in single precision (section 2.4: the binary32
 * constants nu = FLT_MAX, fl(sqrt nu) = 1.844674297E+19, mu = FLT_TRUE_MIN,
 * eta = FLT_MAX_EXP - 4; every operation in binary32, round to nearest).
 * Streams as above with float in place of double; zeta' in [-273, 3].
 * Errors as above. */
typedef struct {
  const float *a11, *a22, *a21_re, *a21_im;
  float *cos_phi, *ea_tan_re, *ea_tan_im;
  float *lambda1, *lambda2;
  int32_t *zeta_p;
} jsvd_evd2_streams_f32;

JSVD_API int jsvd_evd2x2_batched_f32(jsvd_field field, const jsvd_evd2_streams_f32 *s, int64_t n,
                                     void *stream);

/* The same batched EVD on HOST streams (same meaning and rules as above,
 * every pointer in *s a host pointer), by the kernel of
 * jsvd_evd2x2_batched (same bits).  When every stream is page-locked memory
 * mapped for the current device (cudaHostAlloc, pinned tensors), the
 * kernel reads and writes the streams in place over the host link, with no
 * staging.  Otherwise (or with JSVD_TUNE_EVD_HOST = 1) the batch is cut
 * into chunks that are copied to `work`, transformed and copied back, three
 * chunks in flight on internal streams of the current device.  The call is
 * asynchronous on `stream` like the others: the outputs are complete once
 * `stream` has reached this point.  Pageable buffers give the same results
 * with the copies serialised.  work: DEVICE, 256-byte aligned,
 * jsvd_evd2x2_host_workspace_size bytes, not used by anything else until
 * `stream` passes this call.  Errors: as above, -4 work NULL or misaligned,
 * JSVD_E_WORKSPACE if work_bytes is too small. */
JSVD_API int jsvd_evd2x2_host_workspace_size(size_t *bytes);
JSVD_API int jsvd_evd2x2_batched_host(jsvd_field field, const jsvd_evd2_streams *s, int64_t n,
                                      void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Wide-exponent Frobenius norms of the columns of A (supplement SM6,
 * Alg. rnF): ||a_j|| = 2^e_j f_j with e_j integral (returned as a double,
 * -inf for a zero column) and f_j in [1, 2), computed without overflow or
 * underflow of any partial sum (the norm of a column of FLT/DBL_MAX entries
 * or of subnormals is accurate).  A: m x n column-major, lda >= m; complex
 * A interleaved (each row adds Re^2 then Im^2).  The order of the sums is
 * fixed by m: L = 32 lanes for m <= 8192, else 1024; lane t adds rows t,
 * t+L, ... in order, and the lanes are combined by the xor butterfly within
 * each group of 32 and then (L = 1024) over the 32 groups, so the bits do
 * not depend on the launch.  e_out, f_out: n
 * doubles each (device).  Errors: -1 field, -2 m < 0, -3 n < 0, -4 A NULL,
 * -5 lda, -6 e_out or f_out NULL. */
JSVD_API int jsvd_colnorm_ef(jsvd_field field, int64_t m, int64_t n, const void *A, int64_t lda,
                             double *e_out, double *f_out, void *stream);

/* ------------------------------------------------------------------------
 * One-sided Jacobi SVD (section 4, Alg. zvjsvd; real variant dvjsvd).
 *
 * A = U diag(sigma) V^H for an m x n matrix A, m >= n >= 1, by repeated
 * parallel steps: for every pivot pair (p, q) of a cyclic parallel ordering
 * (n/2 disjoint pairs per step, n-1 steps per sweep; the round-robin
 * ordering, a phantom column added for odd n -- section 4.1), the column
 * norms and the scaled dot-product g_q^* g_p / (||g_p|| ||g_q||)
 * (Alg. zdpscl), the convergence test |a21'| >= fl(eps sqrt(m)),
 * eps = 2^-53 (Eq. e:tol, Alg. cvg), the scaled Grammian (Alg. Gram), its
 * 2x2 EVD (as jsvd_evd2x2_batched) and the transformation of the column pair
 * of G and of V (Eq. e:transf, Alg. zjrot).  With opts->permute the pair is
 * transformed by U P, the columns swapped when the EVD's permutation bit says
 * so (section 2; optional there, and with the round-robin ordering it more
 * than doubles the sweep count, so it is off by default: the columns are
 * sorted once after convergence instead).  Sweeps stop when a whole sweep
 * performs no rotation (section 3.3.1), or after opts->max_sweeps.  The
 * iteration matrix is kept at a power-of-two scale with max-norm in [1, 2)
 * and rescaled if it grows past 2^opts->rescale_exp (section 3.2); the
 * singular values are returned unscaled, also as (e, f) pairs,
 * sigma = 2^e f, 1 <= f < 2 (section 4.2.1), sorted non-increasingly with the
 * columns of U and V permuted alike.
 *
 * Layout: column-major.  JSVD_REAL: A, U, V are double.  JSVD_COMPLEX: A, U,
 * V are interleaved complex double (re, im), lda/ldu/ldv counted in complex
 * elements; the library splits them into separate planes internally
 * (section 2.4.1, supplement SM5).
 */
#define JSVD_FP64 0
#define JSVD_MIXED_FP32_FP64 1

typedef struct {
  int32_t max_sweeps;  /* S; <= 0 selects the default, 100 */
  int32_t mode;        /* JSVD_FP64 or JSVD_MIXED_FP32_FP64 */
  int32_t rescale_exp; /* R: G starts with ||G||_max in [2^(R-25), 2^(R-24))
                          ([1, 2) for R <= 25) and is scaled back there
                          whenever ||G||_max reaches 2^R (section 3.2);
                          0 selects 480; must be in [1, 480] */
  int32_t permute;     /* 1: apply the column swap P during the sweeps;
                          0 (default): do not */
  int32_t compensated; /* 1: the pivot pairs' dot-products g_q^* g_p by the
                          compensated summation of supplement SM2.2
                          (Alg. zdpscl' / ddpscl': products rounded down
                          plus their exact errors, each stream summed by
                          Kahan's method with 2Sum); FP64 sweeps only.
                          0 (default): plain fma sums (Alg. zdpscl) */
} jsvd_opts;

/* Per-matrix outcome, written to DEVICE memory by the kernels. */
typedef struct {
  int32_t status;    /* 0 = converged; JSVD_NOT_CONVERGED; JSVD_E_NONFINITE
                        (A holds Inf/NaN: outputs are NaN); JSVD_E_TIMEOUT */
  int32_t sweeps;    /* sweeps performed, the last (rotation-free) included */
  int64_t rotations; /* transformations applied in total */
  int32_t rescales;  /* downscalings of the iteration matrix */
  int32_t sweeps_fp32; /* mixed mode: sweeps of the FP32 phase */
  int32_t gs_steps;    /* transformations done as the Gram-Schmidt step of
                          section 3.5.1 (Eq. e:GS: column norms more than
                          2^1023 fl(eps sqrt m) apart), counted in rotations */
  int32_t reserved;
} jsvd_info;

#define JSVD_NOT_CONVERGED 1

/* Bytes of device workspace jsvd_svd needs for these arguments.
 * Errors: -1 field, -2 opts invalid, -3 m, -4 n (m >= n >= 1), -5 bytes NULL. */
JSVD_API int jsvd_svd_workspace_size(jsvd_field field, const jsvd_opts *opts, int64_t m,
                                     int64_t n, size_t *bytes);

/* SVD of one matrix.  opts may be NULL (all defaults).  A is read only; U
 * (m x n, ldu >= m), sigma (n), V (n x n, ldv >= n) are written; sigma_e,
 * sigma_f (n doubles each) and info may be NULL.  work must be 256-byte
 * aligned and hold jsvd_svd_workspace_size bytes; its contents on entry do
 * not matter.  Errors: -i for argument i, JSVD_E_WORKSPACE,
 * JSVD_E_UNSUPPORTED (the sweep kernel cannot be made resident: zero blocks
 * per SM), JSVD_E_CUDA (also when the device's SM count cannot be read). */
JSVD_API int jsvd_svd(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                      const void *A, int64_t lda, void *U, int64_t ldu, double *sigma,
                      double *sigma_e, double *sigma_f, void *V, int64_t ldv, void *work,
                      size_t work_bytes, jsvd_info *info, void *stream);

/* The SVD of a single precision matrix (float; complex: interleaved float
 * pairs): FP32 columns updated by Eq. e:transf, each pivot pair's lane sums
 * combined in FP64 and its rotation taken from the FP64 2x2 EVD, the final
 * norms in FP64; converged when no pair has |a21'| >= fl(eps sqrt m),
 * eps = 2^-24 (Eq. e:tol in single precision).  Outputs in single
 * precision: U (m x n, ldu >= m), sigma (n floats, non-increasing), V
 * (n x n, ldv >= n).  opts as for jsvd_svd (mode and rescale_exp are not
 * used; compensated must be 0).  work: jsvd_svd_f32_workspace_size bytes,
 * 256-byte aligned.  Errors: -1 field, -2 opts, -3 m, -4 n, -5 A, -6 lda,
 * -7 U, -8 ldu, -9 sigma, -10 V, -11 ldv, -12 work, JSVD_E_WORKSPACE,
 * JSVD_E_UNSUPPORTED, JSVD_E_CUDA. */
JSVD_API int jsvd_svd_f32_workspace_size(jsvd_field field, const jsvd_opts *opts, int64_t m,
                                         int64_t n, size_t *bytes);
JSVD_API int jsvd_svd_f32(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                          const void *A, int64_t lda, void *U, int64_t ldu, float *sigma, void *V,
                          int64_t ldv, void *work, size_t work_bytes, jsvd_info *info,
                          void *stream);

/* ------------------------------------------------------------------------
 * Batched SVD of many matrices of uneven sizes: the same computation as
 * jsvd_svd for each matrix (bit for bit), in one persistent launch whose
 * blocks take whole matrices from a queue ordered longest first.  The
 * descriptor arrays (m, n, A, lda, U, ldu, sigma, sigma_e, sigma_f, V, ldv;
 * count entries each) are HOST arrays; the matrices they point to are
 * device memory, laid out as for jsvd_svd.  sigma_e and sigma_f may be
 * NULL (not wanted).  info is a DEVICE array of count jsvd_info (may be
 * NULL).  opts->mode must be JSVD_FP64.
 *
 * jsvd_svd_batched = jsvd_svd_batched_prepare + jsvd_svd_batched_launch.
 * prepare copies the descriptors into work (it returns after the copy is
 * done, so the host arrays may then be reused); launch only enqueues device
 * work (a memset and one kernel) and may be repeated on the same prepared
 * workspace, e.g. as a captured CUDA graph.
 * Errors: -i for argument i (-4 also for an invalid m[i] or n[i], -6 for
 * an invalid A[i]/lda[i], -8 U[i]/ldu[i], -10 sigma[i], -13 V[i]/ldv[i]),
 * JSVD_E_WORKSPACE, JSVD_E_CUDA. */
JSVD_API int jsvd_svd_batched_workspace_size(jsvd_field field, const jsvd_opts *opts,
                                             int64_t count, const int64_t *m, const int64_t *n,
                                             size_t *bytes);
JSVD_API int jsvd_svd_batched_prepare(jsvd_field field, const jsvd_opts *opts, int64_t count,
                                      const int64_t *m, const int64_t *n, const void *const *A,
                                      const int64_t *lda, void *const *U, const int64_t *ldu,
                                      double *const *sigma, double *const *sigma_e,
                                      double *const *sigma_f, void *const *V, const int64_t *ldv,
                                      void *work, size_t work_bytes, void *stream);
JSVD_API int jsvd_svd_batched_launch(jsvd_field field, const jsvd_opts *opts, int64_t count,
                                     void *work, jsvd_info *info, void *stream);
JSVD_API int jsvd_svd_batched(jsvd_field field, const jsvd_opts *opts, int64_t count,
                              const int64_t *m, const int64_t *n, const void *const *A,
                              const int64_t *lda, void *const *U, const int64_t *ldu,
                              double *const *sigma, double *const *sigma_e, double *const *sigma_f,
                              void *const *V, const int64_t *ldv, void *work, size_t work_bytes,
                              jsvd_info *info, void *stream);

/* ------------------------------------------------------------------------
 * The SVD adjoint (not in the paper; the differentiated form of the SVD):
 * for count real matrices A_b = U_b diag(s_b) V_b^T (m x n, m >= n, distinct
 * singular values) and cotangents Ubar_b, sbar_b, Vbar_b, computes
 *   Abar = U [(F o (U^T Ubar - Ubar^T U)) S + diag(sbar)
 *             + S (F o (V^T Vbar - Vbar^T V))] V^T + (I - U U^T) Ubar S^-1 V^T,
 *   F_ij = 1/(s_j^2 - s_i^2) (i != j), 0 on the diagonal
 * (Townsend 2016).  All arrays are DEVICE memory, packed: matrix b of U,
 * Ubar, Abar (m x n, column-major, ld = m) at b m n, of V, Vbar (n x n) at
 * b n n, of s, sbar at b n.  Ubar, sbar, Vbar may be NULL (zero).  One
 * block per matrix with its operands in shared memory: needs
 * 8 (3 m n + 4 n n) <= 200 KiB (else JSVD_E_UNSUPPORTED).
 * Errors: -i for argument i, JSVD_E_UNSUPPORTED, JSVD_E_CUDA. */
JSVD_API int jsvd_svd_adjoint_batched(int64_t count, int64_t m, int64_t n, const double *U,
                                      const double *s, const double *V, const double *Ubar,
                                      const double *sbar, const double *Vbar, double *Abar,
                                      void *stream);

/* Sign gauge of real singular vectors: flips each pair (u_j, v_j) of the
 * count packed matrices (layout as above) so that the entry of largest
 * magnitude of u_j is positive (the first such entry on ties).  Makes U and
 * V functions of A wherever the singular values are distinct, as a
 * differentiated loss on U needs.  Errors: -i for argument i, JSVD_E_CUDA. */
JSVD_API int jsvd_sign_gauge_batched(int64_t count, int64_t m, int64_t n, double *U, double *V,
                                     void *stream);

/* jsvd_svd for callers that cannot allocate device memory at run time --
 * for instance code inside a framework whose caching allocator already holds
 * the GPU's memory (another cudaMalloc may fail there), latency-critical
 * loops that cannot afford cudaMalloc's implicit synchronisation, or
 * processes whose memory footprint is fixed at start-up.  The paper has no
 * counterpart; it is the same computation as jsvd_svd.
 *
 * It takes no workspace and allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call).  Its scratch is one static device array of
 * JSVD_NOALLOC_SCRATCH_BYTES (16 MiB) inside the library, which every GPU
 * that loads the library keeps until the process exits.  A problem fits
 * when jsvd_svd_workspace_size, called with the same field and opts, is at
 * most that; otherwise it is rejected with JSVD_E_WORKSPACE.  The mixed
 * mode needs more scratch than plain FP64.  Examples: in JSVD_FP64 real
 * 2048 x 512 and complex 512 x 512 fit, real 1024 x 1024 does not; in
 * JSVD_MIXED_FP32_FP64 real 512 x 512 and complex 384 x 384 fit, real
 * 1024 x 512 and complex 512 x 512 do not.
 *
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, a host-side query; the first call in a context may
 * load the library's device code there, so make it before any stream
 * capture).  The address is not cached, so calls stay correct after
 * cudaDeviceReset or a change of the current context.  All calls share the
 * one array and it keeps the last call's contents: each call clears the
 * state that must start at zero, but calls whose work overlaps on the GPU
 * (different streams, or different host threads) race on it and give wrong
 * results -- serialise them.
 *
 * Arguments and results as jsvd_svd, without work/work_bytes; A, U, sigma,
 * V (and the optional sigma_e, sigma_f, info) remain the caller's device
 * buffers.  Errors: -i for argument i (1..13), JSVD_E_WORKSPACE when the
 * problem does not fit the scratch, JSVD_E_UNSUPPORTED when the sweep
 * kernel cannot be made resident on the device (an occupancy of zero
 * blocks per SM), JSVD_E_CUDA. */
#define JSVD_NOALLOC_SCRATCH_BYTES (16u << 20)
JSVD_API int jsvd_svd_noalloc(jsvd_field field, const jsvd_opts *opts, int64_t m, int64_t n,
                              const void *A, int64_t lda, void *U, int64_t ldu, double *sigma,
                              double *sigma_e, double *sigma_f, void *V, int64_t ldv,
                              jsvd_info *info, void *stream);

/* C = alpha op(A) B + beta C for column-major FP64 matrices on the FP64
 * tensor path (mma.sync m8n8k4 f64): the dense products of the mixed SVD
 * (G = A V0 and the Newton-Schulz re-orthogonalisation of V).  op(A) = A
 * (M x K, lda >= M) for transA == 0, A^T (A stored K x M, lda >= K) for
 * transA == 1; B is K x N (ldb >= K); C is M x N (ldc >= M) and must not
 * overlap A or B.  M, N or K = 0 is allowed (K = 0 scales C by beta).
 * Errors: -i for argument i, JSVD_E_CUDA. */
JSVD_API int jsvd_dgemm(int transA, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                        double *C, int64_t ldc, void *stream);

/* Complex C = alpha op(A) B + beta C on split planes (real and imaginary
 * parts each a column-major FP64 matrix with the same leading dimension),
 * on the same tensor path by the 3M form: T1 = op(Ar) Br, T2 = op(Ai) Bi,
 * T3 = op(Ar +- Ai)(Br + Bi) give Re = T1 -+ T2 and Im = (T3 - T1) -+ T2,
 * three real products in place of four.  The mixed SVD's complex products
 * (G = A V0, Newton-Schulz on V) use it.  op(A) = A (M x K, lda >= M) for
 * transA == 0, the conjugate transpose A^H (A stored K x M, lda >= K) for
 * transA == 1; B is K x N (ldb >= K); C is M x N (ldc >= M) and must not
 * overlap A or B.  Each entry's imaginary part carries an error of order
 * K eps (|Ar| + |Ai|)(|Br| + |Bi|).  herm == 1 computes the Hermitian
 * C = alpha A^H A: it requires transA == 1, N == M, Br == Ar, Bi == Ai,
 * ldb == lda and beta == 0, forms only the tiles on and above the diagonal,
 * writes both triangles (C == C^H exactly) and a zero imaginary diagonal.
 * M, N or K = 0 is allowed.  Errors: -i for argument i, JSVD_E_CUDA. */
JSVD_API int jsvd_zgemm(int transA, int herm, int64_t M, int64_t N, int64_t K, double alpha,
                        const double *Ar, const double *Ai, int64_t lda, const double *Br,
                        const double *Bi, int64_t ldb, double beta, double *Cr, double *Ci,
                        int64_t ldc, void *stream);

/* Self-test of the library's integer-pipe binary64 division and square
 * root (both their branching and their select-based forms) against the
 * GPU's IEEE FP64 instructions: n generated operand pairs
 * (several families: arbitrary bit patterns, subnormals, powers of two,
 * extremes), from seed; atomically ADDS the number of differing divisions
 * to mismatches[0] and of square roots to mismatches[1] (DEVICE memory, two
 * unsigned long long, zeroed by the caller).  Errors: -i, JSVD_E_CUDA. */
/* Self-test of the branch-free binary32 division of the single precision
 * EVD (JSVD_TUNE_EVD32_DIV = 1) against the GPU's IEEE FP32 division: n
 * generated operand pairs (arbitrary bit patterns, subnormals, powers of
 * two, extremes, zeros), from seed; atomically ADDS the number of results
 * whose bits differ (two NaNs count as equal) to *mismatches (DEVICE, one
 * unsigned long long, zeroed by the caller).  Errors: -1 n < 0,
 * -3 mismatches NULL, JSVD_E_CUDA. */
JSVD_API int jsvd_selftest_fp32div(int64_t n, uint64_t seed, unsigned long long *mismatches,
                                   void *stream);

JSVD_API int jsvd_selftest_fp64(int64_t n, uint64_t seed, unsigned long long *mismatches,
                                void *stream);

/* Throughput probe of the FP64 pipe, the measured denominator of an
 * FP64-pipe roofline (the paper has no counterpart): `blocks` blocks of
 * `threads` threads (32 .. 256, a multiple of 32), each thread 8
 * independent chains of `iters` operations of one kind -- 0: fused
 * multiply-add (lane operations = blocks * threads * 8 * iters); 1: the IEEE
 * square root; 2: the IEEE division.  With many blocks the pipe's
 * throughput sets the time; with one block of 32 threads, one warp's FP64
 * issue rate.  The caller times the launch on `stream`.  sink: one DEVICE
 * double the kernel writes.  Errors: -1 kind, -2 iters < 1, -3 blocks < 1,
 * -4 threads, -5 sink NULL, JSVD_E_CUDA. */
JSVD_API int jsvd_probe_fp64_rate(int kind, int64_t iters, int blocks, int threads,
                                  double *sink, void *stream);

/* Failure-detection self-test of the bounded grid barrier the persistent
 * SVD kernel uses between steps: a cooperative launch of `blocks` blocks
 * (1 .. number of SMs) takes `rounds` barriers; block `absent` (-1: none)
 * never arrives, so the others' wait gives up after limit_ns (1e6 .. 5e9)
 * and they stop.  status (DEVICE, 2 int32): [0] = JSVD_E_TIMEOUT if a wait
 * gave up, else JSVD_OK; [1] = barriers completed over all blocks.  The
 * context stays usable.  Errors: -1 blocks, -3 rounds, -4 limit_ns,
 * -5 status NULL, JSVD_E_CUDA.  Concurrent calls share one state. */
JSVD_API int jsvd_selftest_barrier(int blocks, int absent, int rounds, int64_t limit_ns,
                                   int32_t *status, void *stream);

/* The parallel pivot ordering the SVD kernels use (section 4.1; the
 * round-robin reading): writes (nt - 1) x (nt / 2) pairs (p, q), p < q, as
 * int32 [step][pair][2] into the DEVICE buffer tab, nt = n + (n & 1) (a
 * phantom column n for odd n), computed by the same device function the
 * sweeps use.  Errors: -1 n < 2, -2 tab NULL, JSVD_E_CUDA. */
JSVD_API int jsvd_ordering(int32_t n, int32_t *tab, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* JSVD_H */

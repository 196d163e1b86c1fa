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

/* Library version as 10000*major + 100*minor + patch. */
JSVD_API int jsvd_version(void);

/* Static description of a return code (never NULL). */
JSVD_API const char *jsvd_strerror(int code);

/* Text of the last CUDA error this host thread saw (after JSVD_E_CUDA). */
JSVD_API const char *jsvd_last_cuda_error(void);

/* Launch-shape knobs.  They are arithmetic-neutral: no setting changes a
 * single result bit, only the speed.  Process-wide; returns -2 or -3 for a
 * value out of range, -1 for an unknown knob.
 *   JSVD_TUNE_EVD_LAUNCH: value = threads per block of the 2x2 EVD kernel
 *     (64, 128 or 256), value2 = resident blocks per SM (1..64). */
#define JSVD_TUNE_EVD_LAUNCH 1
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

#ifdef __cplusplus
}
#endif

#endif /* JSVD_H */

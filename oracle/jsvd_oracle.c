/*
 * jsvd_oracle.c -- the CPU oracle of the Jacobi SVD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, scalar FP64
 * restatement of Novakovic, "Vectorization of a thread-parallel Jacobi
 * singular value decomposition method" (arXiv 2202.08361).  It shares no
 * code, header, table or constant generator with the CUDA library; only
 * tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * it.  The product path never calls it.
 *
 * Contents (each function cites the passage it follows):
 *   orc_dsjac2 / orc_zsjac2  batched 2x2 real symmetric / complex Hermitian
 *                            EVD, restated from the equations of section 2
 *                            (Eq. "e:z", "e:zpolar", "e:tan2", "e:jactan",
 *                            "e:jacsec", "e:lamsec"), one matrix at a time,
 *                            with the rounded operations of Alg. d8jac2 /
 *                            z8jac2 in their order.
 *   orc_ssjac2 / orc_csjac2  the same in single precision with the
 *                            binary32 constants of section 2.4.
 *   orc_pairs                the cyclic parallel pivot ordering (round-robin
 *                            reading of section 4.1).
 *   orc_vjsvd                one-sided Jacobi SVD after Alg. zvjsvd
 *                            (section 4.3), real or complex (split planes),
 *                            with the rescaling heuristic of section 3.2
 *                            (its threshold lowerable for the tests),
 *                            the scaled dot-products of Alg. zdpscl
 *                            (section 3.3) or, optionally, Alg. zdpscl' /
 *                            ddpscl' (compensated, supplement SM2.2),
 *                            the convergence test of Eq.
 *                            "e:tol", the scaled Grammians of Alg. Gram
 *                            (section 3.4) and the transformations of
 *                            Eq. "e:transf" / Alg. zjrot (section 3.5).
 *   orc_rnF                  the wide-exponent Frobenius norm of Alg. rnF
 *                            (supplement SM6) with one lane.
 *   orc_svd_adjoint          thin real SVD adjoint (Townsend 2016), used for
 *                            the differentiated batched SVD.
 *
 * Compile with -ffp-contract=off: every fused multiply-add below is an
 * explicit fma() call, exactly where the paper writes one.
 *
 * Readings of the paper where it is silent:
 *   - zeta of an all-zero 2x2 matrix follows section 2.3.1 (frexp of the
 *     smallest subnormal), so zeta is a finite int in [-3, 2094];
 *   - the packed (zeta' << 1) | p is formed by an unsigned shift;
 *   - the column swap P of section 2 (Alg. zvjsvd: U P) is optional, as
 *     section 2 needs it only when the transformed pivot columns must also
 *     come out sorted by norm: with permute != 0 the EVD is computed for every pivot
 *     pair, a rotated pair is transformed by U P and a pair that is not
 *     rotated is swapped iff its EVD says lambda1' < lambda2'; with
 *     permute == 0 (the default) no column moves during the sweeps -- with
 *     the round-robin ordering, P more than doubles the sweep count;
 *   - a pair with a zero column is never rotated; with permute != 0 it is
 *     swapped iff the norm of g_p is below that of g_q;
 *   - column norms are computed by a two-pass, overflow-free scaled sum of
 *     squares (max-exponent prescaling), standing in for xNRM2; the norm
 *     overflow branch of Alg. zvjsvd therefore never fires;
 *   - odd n: a phantom column n is added to the ordering and pairs that
 *     contain it are skipped;
 *   - after convergence the singular values are sorted non-increasingly
 *     (stable), permuting the columns of U and V alike.
 */
#include <float.h>
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* Mutation points for the tests that check the pins (tests/
 * test_oracle_mutants.py): compiled with -DORC_MUTANT=k (k > 0), MUT(k, ...)
 * takes its second expression, a planted mistake; by default (0) every
 * MUT is its first expression and the code is the plain oracle. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#define MUT(k, good, bad) ((ORC_MUTANT == (k)) ? (bad) : (good))

/* Threads of a parallel loop: nthreads if positive, else the default. */
static int omp_threads(int nthreads)
{
#ifdef _OPENMP
  return (nthreads > 0) ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * The 2x2 Hermitian EVD of section 2, restated from its equations:
 *   Eq. "e:z"       the power-of-two scaling A' = 2^zeta A;
 *   Eq. "e:zpolar"  the polar form |a21| e^{i alpha} of a21 (complex), with
 *                   |a21| from Alg. hypot (Eq. "e:hypot");
 *   Eq. "e:tan2", "e:jactan", "e:jacsec", "e:lamsec"   the rotation and
 *                   the eigenvalues of section 2.1.
 * Every rounded operation below is one the equations write, in their
 * order, so the results are those of Alg. d8jac2 / z8jac2 lane by lane. */

/* floor(lg x) for finite x > 0 (the AVX-512 getexp; subnormals too). */
static int flg(double x)
{
  int e;
  (void)frexp(x, &e);
  return e - 1;
}

static int imin(int a, int b) { return (a <= b) ? a : b; }

/* nu, the largest finite value, and mu-check, the smallest positive
 * subnormal (section 2.2). */
#define NU DBL_MAX
#define MU_CHECK DBL_TRUE_MIN

/* zeta_x of Eq. "e:z": eta - floor(lg|x|) with eta = floor(lg(nu/8)) =
 * 1020.  lg 0 is read as lg mu-check (the serial scaling of section 2.3.1),
 * so an all-zero matrix gets the finite zeta = 1020 + 1074 = 2094. */
static int zeta_elem(double x)
{
  const int eta = flg(NU / 8.0) + MUT(5, 0, 1);
  return eta - flg(fmax(fabs(x), MU_CHECK));
}

/* x sign(s), sign(+-0) = +-1: the sign bit of s XOR-ed into x, exact (the
 * sign transfer Alg. d8jac2 applies to tan(phi)). */
static double xorsign(double x, double s)
{
  uint64_t a, b;
  memcpy(&a, &x, 8);
  memcpy(&b, &s, 8);
  a ^= (b & 0x8000000000000000ull);
  memcpy(&x, &a, 8);
  return x;
}

/* Alg. hypot: sqrt(x^2 + y^2) = M sqrt(q^2 + 1), q = m / M, m and M the
 * smaller and larger of |x|, |y| (Eq. "e:hypot"); fmax(., 0) turns the
 * 0/0 of x = y = 0 into q = 0.  Also the |z| of Alg. cvg. */
static double hypot_naive(double x, double y)
{
  const double ax = fabs(x), ay = fabs(y);
  const double m = fmin(ax, ay), M = fmax(ax, ay);
  const double q = fmax(m / M, 0.0);
  return sqrt(fma(q, q, 1.0)) * M;
}

/* Section 2.1 for an already scaled matrix: only |a21| enters. */
struct jacrot {
  double tan_phi;  /* tan(phi) >= 0 iff a11 - a22 >= 0            */
  double sec2_phi; /* sec^2(phi)                                   */
  double cos_phi;  /* 1 / sec(phi)                                 */
  double lam1, lam2; /* the eigenvalues lambda' of the scaled matrix */
};

static void jacobi_rotation(double a11, double a22, double abs_a21, struct jacrot *J)
{
  /* Eq. "e:tan2": tan(2phi) = min(fmax(2|a21| / |a|, 0), fl(sqrt nu)) sign a
   * with a = a11 - a22.  2|a21| is exact; fmax sends 0/0 to 0, so the min
   * never sees a NaN; the sign of a is copied in, an exact multiply by +-1. */
  const double two_abs_a21 = 2.0 * abs_a21;
  const double a = a11 - a22;
  const double tan_2phi = copysign(fmin(fmax(two_abs_a21 / fabs(a), 0.0), sqrt(NU)), a);
  /* Eq. "e:jactan" */
  const double t = tan_2phi / (1.0 + sqrt(fma(tan_2phi, tan_2phi, 1.0)));
  /* Eq. "e:jacsec": sec^2 = fma(tan, tan, 1), sec = sqrt(sec^2), cos = 1/sec */
  const double sec2 = fma(t, t, 1.0);
  J->tan_phi = t;
  J->sec2_phi = sec2;
  J->cos_phi = MUT(2, 1.0 / sqrt(sec2), 1.0 / sec2);
  /* Eq. "e:lamsec": lambda_1 = ((a22 tan + 2|a21|) tan + a11) / sec^2,
   *                 lambda_2 = ((a11 tan - 2|a21|) tan + a22) / sec^2 */
  J->lam1 = fma(fma(MUT(1, a22, a11), t, two_abs_a21), t, a11) / sec2;
  J->lam2 = fma(fma(a11, t, -two_abs_a21), t, a22) / sec2;
}

/* What one EVD returns (section 2.3): cos(phi), e^{i alpha} tan(phi), the
 * backscaled eigenvalues lambda = 2^-zeta lambda', the scaled lambda', zeta
 * and the permutation bit p = (lambda1' < lambda2'). */
struct evd2 {
  double cos_phi, eatan_re, eatan_im;
  double lam1, lam2, lam1s, lam2s;
  int zeta, p;
};

static void evd2_finish(const struct jacrot *J, int zeta, struct evd2 *o)
{
  o->cos_phi = J->cos_phi;
  o->lam1s = J->lam1;
  o->lam2s = J->lam2;
  o->lam1 = scalbn(J->lam1, -zeta);
  o->lam2 = scalbn(J->lam2, -zeta);
  o->zeta = zeta;
  o->p = (J->lam1 < J->lam2);
}

/* Real symmetric EVD (Alg. d8jac2, one lane): e^{i alpha} = sign a21. */
static void evd2_real(double a11, double a22, double a21, struct evd2 *o)
{
  const int zeta = imin(imin(zeta_elem(a11), zeta_elem(a22)), zeta_elem(a21));
  a11 = scalbn(a11, zeta);
  a22 = scalbn(a22, zeta);
  a21 = scalbn(a21, zeta);
  struct jacrot J;
  jacobi_rotation(a11, a22, fabs(a21), &J);
  o->eatan_re = MUT(3, xorsign(J.tan_phi, a21), J.tan_phi);
  o->eatan_im = 0.0;
  evd2_finish(&J, zeta, o);
}

/* Complex Hermitian EVD (Alg. z8jac2, one lane). */
static void evd2_complex(double a11, double a22, double a21r, double a21i, struct evd2 *o)
{
  const int zeta = imin(imin(zeta_elem(a11), zeta_elem(a22)),
                        imin(zeta_elem(a21r), zeta_elem(a21i)));
  a11 = scalbn(a11, zeta);
  a22 = scalbn(a22, zeta);
  a21r = scalbn(a21r, zeta);
  a21i = scalbn(a21i, zeta);
  /* Eq. "e:zpolar": cos(alpha) = fmin(|Re a21| / |a21|, 1) sign(Re a21),
   * sin(alpha) = Im a21 / max(|a21|, mu-check) */
  const double abs_a21 = hypot_naive(a21r, a21i);
  const double cos_alpha = copysign(fmin(fabs(a21r) / abs_a21, 1.0), a21r);
  const double sin_alpha = MUT(4, a21i, -a21i) / fmax(abs_a21, MU_CHECK);
  struct jacrot J;
  jacobi_rotation(a11, a22, abs_a21, &J);
  o->eatan_re = cos_alpha * J.tan_phi;
  o->eatan_im = sin_alpha * J.tan_phi;
  evd2_finish(&J, zeta, o);
}

/* Pack (zeta' << 1) | p, zeta' = -zeta, through an unsigned shift (a
 * negative int may not be left-shifted in C). */
static int32_t pack_zp(int zeta, int p)
{
  uint32_t u = ((uint32_t)(-zeta)) << 1;
  return (int32_t)(u | (uint32_t)(p != 0));
}

/* Batched real EVD (Alg. dbjac2): outputs cos(phi), sign(a21) tan(phi),
 * lambda1, lambda2 and the packed (zeta', p); lam1, lam2, zp may be NULL. */
ORC_EXPORT void orc_dsjac2(int64_t r, const double *a11, const double *a22, const double *a21,
                           double *cphi, double *tphi, double *lam1, double *lam2, int32_t *zp,
                           int nthreads)
{
#pragma omp parallel for schedule(static) num_threads(omp_threads(nthreads))
  for (int64_t i = 0; i < r; ++i) {
    struct evd2 o;
    evd2_real(a11[i], a22[i], a21[i], &o);
    cphi[i] = o.cos_phi;
    tphi[i] = o.eatan_re;
    if (lam1) lam1[i] = o.lam1;
    if (lam2) lam2[i] = o.lam2;
    if (zp) zp[i] = pack_zp(o.zeta, o.p);
  }
}

/* Batched complex EVD (Alg. zbjac2): outputs cos(phi), cos(alpha) tan(phi),
 * sin(alpha) tan(phi), lambda1, lambda2 and the packed (zeta', p). */
ORC_EXPORT void orc_zsjac2(int64_t r, const double *a11, const double *a22, const double *a21r,
                           const double *a21i, double *cphi, double *catphi, double *satphi,
                           double *lam1, double *lam2, int32_t *zp, int nthreads)
{
#pragma omp parallel for schedule(static) num_threads(omp_threads(nthreads))
  for (int64_t i = 0; i < r; ++i) {
    struct evd2 o;
    evd2_complex(a11[i], a22[i], a21r[i], a21i[i], &o);
    cphi[i] = o.cos_phi;
    catphi[i] = o.eatan_re;
    satphi[i] = o.eatan_im;
    if (lam1) lam1[i] = o.lam1;
    if (lam2) lam2[i] = o.lam2;
    if (zp) zp[i] = pack_zp(o.zeta, o.p);
  }
}

/* The scaled eigenvalues lambda' (before backscaling) of the complex EVD,
 * for the pins. */
ORC_EXPORT void orc_zsjac2_scaled(int64_t r, const double *a11, const double *a22,
                                  const double *a21r, const double *a21i, double *lam1s,
                                  double *lam2s)
{
  for (int64_t i = 0; i < r; ++i) {
    struct evd2 o;
    evd2_complex(a11[i], a22[i], a21r[i], a21i[i], &o);
    lam1s[i] = o.lam1s;
    lam2s[i] = o.lam2s;
  }
}

/* ------------------------------------------------------------------------
 * The same EVD in single precision (section 2.4): nu = FLT_MAX, mu-check =
 * FLT_TRUE_MIN, eta = floor(lg(nu/8)) = 124, every operation in binary32.
 * The steps are those of the binary64 functions above. */
#define NU_F FLT_MAX
#define MU_CHECK_F FLT_TRUE_MIN

static int flgf(float x)
{
  int e;
  (void)frexpf(x, &e);
  return e - 1;
}

static int zeta_elem_f(float x)
{
  const int eta = flgf(NU_F / 8.0f);
  return eta - flgf(fmaxf(fabsf(x), MU_CHECK_F));
}

static float xorsignf_(float x, float s)
{
  uint32_t a, b;
  memcpy(&a, &x, 4);
  memcpy(&b, &s, 4);
  a ^= (b & 0x80000000u);
  memcpy(&x, &a, 4);
  return x;
}

static float hypot_naive_f(float x, float y)
{
  const float ax = fabsf(x), ay = fabsf(y);
  const float m = fminf(ax, ay), M = fmaxf(ax, ay);
  const float q = fmaxf(m / M, 0.0f);
  return sqrtf(fmaf(q, q, 1.0f)) * M;
}

struct jacrot_f {
  float tan_phi, sec2_phi, cos_phi, lam1, lam2;
};

static void jacobi_rotation_f(float a11, float a22, float abs_a21, struct jacrot_f *J)
{
  const float two_abs_a21 = 2.0f * abs_a21;                                /* Eq. "e:tan2" */
  const float a = a11 - a22;
  const float tan_2phi = copysignf(fminf(fmaxf(two_abs_a21 / fabsf(a), 0.0f), sqrtf(NU_F)), a);
  const float t = tan_2phi / (1.0f + sqrtf(fmaf(tan_2phi, tan_2phi, 1.0f))); /* "e:jactan" */
  const float sec2 = fmaf(t, t, 1.0f);                                       /* "e:jacsec" */
  J->tan_phi = t;
  J->sec2_phi = sec2;
  J->cos_phi = MUT(13, 1.0f / sqrtf(sec2), 1.0f / sec2);
  J->lam1 = fmaf(fmaf(a22, t, two_abs_a21), t, a11) / sec2;                   /* "e:lamsec" */
  J->lam2 = fmaf(fmaf(a11, t, -two_abs_a21), t, a22) / sec2;
}

ORC_EXPORT void orc_ssjac2(int64_t r, const float *a11, const float *a22, const float *a21,
                           float *cphi, float *tphi, float *lam1, float *lam2, int32_t *zp)
{
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < r; ++i) {
    const int zeta = imin(imin(zeta_elem_f(a11[i]), zeta_elem_f(a22[i])), zeta_elem_f(a21[i]));
    const float b11 = scalbnf(a11[i], zeta), b22 = scalbnf(a22[i], zeta);
    const float b21 = scalbnf(a21[i], zeta);
    struct jacrot_f J;
    jacobi_rotation_f(b11, b22, fabsf(b21), &J);
    cphi[i] = J.cos_phi;
    tphi[i] = xorsignf_(J.tan_phi, b21);
    if (lam1) lam1[i] = scalbnf(J.lam1, -zeta);
    if (lam2) lam2[i] = scalbnf(J.lam2, -zeta);
    if (zp) zp[i] = pack_zp(zeta, J.lam1 < J.lam2);
  }
}

ORC_EXPORT void orc_csjac2(int64_t r, const float *a11, const float *a22, const float *a21r,
                           const float *a21i, float *cphi, float *catphi, float *satphi,
                           float *lam1, float *lam2, int32_t *zp)
{
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < r; ++i) {
    const int zeta = imin(imin(zeta_elem_f(a11[i]), zeta_elem_f(a22[i])),
                          imin(zeta_elem_f(a21r[i]), zeta_elem_f(a21i[i])));
    const float b11 = scalbnf(a11[i], zeta), b22 = scalbnf(a22[i], zeta);
    const float br = scalbnf(a21r[i], zeta), bi = scalbnf(a21i[i], zeta);
    const float abs_a21 = hypot_naive_f(br, bi);                               /* "e:zpolar" */
    const float cos_alpha = copysignf(fminf(fabsf(br) / abs_a21, 1.0f), br);
    const float sin_alpha = bi / fmaxf(abs_a21, MU_CHECK_F);
    struct jacrot_f J;
    jacobi_rotation_f(b11, b22, abs_a21, &J);
    cphi[i] = J.cos_phi;
    catphi[i] = cos_alpha * J.tan_phi;
    satphi[i] = sin_alpha * J.tan_phi;
    if (lam1) lam1[i] = scalbnf(J.lam1, -zeta);
    if (lam2) lam2[i] = scalbnf(J.lam2, -zeta);
    if (zp) zp[i] = pack_zp(zeta, J.lam1 < J.lam2);
  }
}

/* ------------------------------------------------------------------------
 * The cyclic parallel ordering.  Section 4.1 asks for a parallel strategy
 * with nt/2 disjoint pairs per step; the MM and ME strategies are defined
 * only in cited work, so the round-robin ("circle") tournament is used:
 * for nt even (nt = n, or n + 1 with a phantom column n when n is odd),
 * step k in [0, nt-1), pair l in [0, nt/2):
 *   l = 0 : (k, nt-1)
 *   l > 0 : {(k + l) mod (nt-1), (k - l) mod (nt-1)}, ordered p < q.
 * Every unordered pair occurs exactly once per sweep.
 * tab receives (nt-1) * (nt/2) * 2 ints, laid out [k][l][p,q].
 * Returns nt. */
ORC_EXPORT int orc_pairs(int n, int32_t *tab)
{
  const int nt = n + (n & 1);
  const int K = nt - 1, L = nt / 2;
  for (int k = 0; k < K; ++k) {
    for (int l = 0; l < L; ++l) {
      int p, q;
      if (l == 0) {
        p = k;
        q = nt - 1;
      } else {
        const int a = (k + l) % K;
        const int b = ((k - l + MUT(8, 0, 1)) % K + K) % K;
        p = (a < b) ? a : b;
        q = (a < b) ? b : a;
      }
      tab[2 * ((int64_t)k * L + l)] = p;
      tab[2 * ((int64_t)k * L + l) + 1] = q;
    }
  }
  return nt;
}

/* ------------------------------------------------------------------------
 * One-sided Jacobi SVD (Alg. zvjsvd, section 4.3). */

/* Return codes shared with tests (not with the library). */
#define ORC_OK 0
#define ORC_E_ARG (-1)
#define ORC_E_NONFINITE (-2)
#define ORC_NOT_CONVERGED 1


/* The Frobenius norm of a column (one or two planes, length m) as (e, f):
 * ||x|| = 2^e f, 1 <= f < 2; zero is (INT_MIN, 1) (section 3.2, the (e,f)
 * representation; supplement SM6.1).  Overflow-free: the column is first
 * divided by 2^E, E the exponent of its max-norm, then the squares are
 * summed in row order with fma. */
static void colnorm(int64_t m, const double *xr, const double *xi, int *e, double *f)
{
  double M = 0.0;
  for (int64_t i = 0; i < m; ++i) M = fmax(M, fabs(xr[i]));
  if (xi)
    for (int64_t i = 0; i < m; ++i) M = fmax(M, fabs(xi[i]));
  if (M == 0.0) {
    *e = INT_MIN;
    *f = 1.0;
    return;
  }
  const int E = flg(M);
  double ssq = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const double y = ldexp(xr[i], -E);
    ssq = fma(y, y, ssq);
  }
  if (xi)
    for (int64_t i = 0; i < m; ++i) {
      const double y = ldexp(xi[i], -E);
      ssq = fma(y, y, ssq);
    }
  /* ||x|| = 2^E sqrt(ssq), 1 <= ssq */
  const double r = sqrt(ssq);
  const int er = flg(r);
  *f = ldexp(r, -er);
  *e = E + er;
}

/* ------------------------------------------------------------------------
 * Alg. rnF (supplement SM6.2-SM6.3) with one lane (s = 1): the Frobenius
 * norm of a vector in the wide-exponent representation r = (e, f) = 2^e f,
 * e an integral double (-inf for zero), f in [1, 2), so that no partial sum
 * overflows or underflows.  Readings: F(0) = 1 (zero is (-inf, 1) as the
 * supplement writes it); scalef by -inf gives 0. */

/* getexp: floor(lg|x|) as a double, -inf for 0 (subnormals normalised) */
static double E_of(double x)
{
  if (x == 0.0) return -INFINITY;
  int e;
  (void)frexp(x, &e);
  return (double)(e - 1);
}

/* getmant to [1, 2): |x| / 2^floor(lg|x|); F(0) = 1 */
static double F_of(double x)
{
  if (x == 0.0) return 1.0;
  int e;
  const double m = frexp(fabs(x), &e); /* [0.5, 1) */
  return 2.0 * m;
}

/* scalef(f, e) for an integral or infinite double e: f 2^e rounded once */
static double scalef_d(double f, double e)
{
  if (e == -INFINITY) return 0.0;
  if (e < -4000.0) e = -4000.0;
  if (e > 4000.0) e = 4000.0;
  return scalbn(f, (int)e);
}

/* One step r <- fma(|x|, |x|, r) in (e, f) arithmetic. */
static void rnf_step(double x, double *e, double *f)
{
  /* r' = r with an even (or infinite) exponent */
  const double lsb = isinf(*e) ? 0.0 : (double)((int64_t)(*e) & 1);
  const double e1 = *e - lsb;
  const double f1 = scalef_d(*f, lsb);
  /* |x| = (E(x), F(x)); x^2 has exponent 2 E(x) or one more */
  const double ex = E_of(x), fx = F_of(x);
  const double eh = 2.0 * ex;
  const double emax = fmax(eh, e1);
  const double dh = fmax(eh - emax, -INFINITY); /* -inf - -inf = NaN -> -inf */
  const double d1 = fmax(e1 - emax, -INFINITY);
  const double fh = scalef_d(fx, dh / 2.0);
  const double fr = scalef_d(f1, d1);
  const double fn = fma(fh, MUT(14, fh, fr), fr);
  *f = F_of(fn);
  *e = emax + E_of(fn);
}

/* (e, f) of ||x||^2 -> (e'', f'') of ||x|| (supplement SM6.1). */
static void ef_sqrt(double e, double f, double *e2, double *f2)
{
  double ep = e, fp = f;
  if (!isinf(e) && ((int64_t)e & 1)) {
    fp = MUT(9, 2.0 * f, f);
    ep = e - 1.0;
  }
  *e2 = isinf(ep) ? ep : ep / 2.0;
  *f2 = sqrt(fp);
}

/* ||x||_F as (e'', f'') by Alg. rnF with one lane. */
ORC_EXPORT void orc_rnF(int64_t m, const double *x, double *e_out, double *f_out)
{
  double e = -INFINITY, f = 1.0;
  for (int64_t i = 0; i < m; ++i) rnf_step(x[i], &e, &f);
  ef_sqrt(e, f, e_out, f_out);
}

/* (e,f) comparison: x < y for norms */
static int ef_less(int ex, double fx, int ey, double fy)
{
  if (ex != ey) return ex < ey;
  return fx < fy;
}

/* Alg. zdpscl: z = fl(g_q^* g_p / (||g_q|| ||g_p||)), the columns prescaled
 * by 2^-e_j in the loop, a single final division by f_q * f_p.  For a real
 * pair qi = pi = NULL and *zi = 0. */
static void zdpscl(int64_t m, const double *qr, const double *qi, const double *pr,
                   const double *pi, int eq, double fq, int ep, double fp, double *zr,
                   double *zi)
{
  double re = 0.0, im = 0.0;
  if (qi) {
    for (int64_t i = 0; i < m; ++i) {
      const double gqr = ldexp(qr[i], -eq), gqi = ldexp(qi[i], -eq);
      const double gpr = ldexp(pr[i], -ep), gpi = ldexp(pi[i], -ep);
      re = fma(gqr, gpr, re);
      im = fma(gqr, gpi, im);
      re = fma(gqi, gpi, re);
      im = fma(MUT(6, -gqi, gqi), gpr, im);
    }
  } else {
    for (int64_t i = 0; i < m; ++i) re = fma(ldexp(qr[i], -eq), ldexp(pr[i], -ep), re);
  }
  const double d = fq * fp;
  *zr = re / d;
  *zi = im / d;
}

/* Eq. "e:d2sum" (2Sum): a + b = s + t exactly, s = fl(a + b). */
static void two_sum(double a, double b, double *s, double *t)
{
  const double ss = a + b;
  double a1 = ss - b;
  double b1 = ss - a1;
  a1 = a - a1;
  b1 = b - b1;
  *s = ss;
  *t = a1 + b1;
}

/* RD(a b), the product rounded toward -infinity.  With p = RN(a b) and its
 * exact residual r = a b - p (one fma), RD(a b) is p when r >= 0 and the
 * next double below p otherwise (RN picks RD or RU). */
static double mul_rd(double a, double b)
{
  const double p = a * b;
  const double r = fma(a, b, -p);
  return (r < 0.0) ? nextafter(p, -INFINITY) : p;
}

/* One term x y of a compensated stream (supplement SM2.2, items G, M and
 * K): c = RD(x y), c' = x y - c >= 0 (one fma), then Kahan's summation with
 * 2Sum on the value stream (s, t) and on the error stream (s', t'). */
static void comp_term(double x, double y, double *s, double *t, double *s2, double *t2)
{
  const double c = mul_rd(x, y);
  const double c2 = fma(x, y, -c);
  two_sum(*s, c + *t, s, t);
  two_sum(*s2, c2 + *t2, s2, t2);
}

/* Alg. zdpscl' (complex) and Alg. ddpscl' (real): the scaled dot-product of
 * Alg. zdpscl with the compensated summation, one stream pair per
 * component, reduced as s + (t + (s' + t')), then one division by
 * f_q f_p.  Reading: the imaginary stream accumulates Re g_q Im g_p -
 * Im g_q Re g_p, the imaginary part of the g_q^* g_p that the algorithm's
 * stated output defines (the printed loop forms its conjugate). */
static void zdpscl_comp(int64_t m, const double *qr, const double *qi, const double *pr,
                        const double *pi, int eq, double fq, int ep, double fp, double *zr,
                        double *zi)
{
  double rs = 0.0, rt = 0.0, rs2 = 0.0, rt2 = 0.0;
  double is = 0.0, it = 0.0, is2 = 0.0, it2 = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const double gqr = ldexp(qr[i], -eq), gpr = ldexp(pr[i], -ep);
    comp_term(gpr, gqr, &rs, &rt, &rs2, &rt2);
    if (qi) {
      const double gqi = ldexp(qi[i], -eq), gpi = ldexp(pi[i], -ep);
      comp_term(gpi, gqi, &rs, &rt, &rs2, &rt2);
      comp_term(gpi, gqr, &is, &it, &is2, &it2);
      comp_term(MUT(17, -gpr, gpr), gqi, &is, &it, &is2, &it2);
    }
  }
  const double d = fq * fp;
  *zr = MUT(10, (rs + (rt + (rs2 + rt2))), (rs + (rs2 + rt2))) / d;
  *zi = qi ? (is + (it + (is2 + it2))) / d : 0.0;
}

/* The scaled dot-product alone (for the tests): z = g_q^* g_p / (2^(e_q +
 * e_p) f_q f_p) by Alg. zdpscl (compensated == 0) or Alg. zdpscl'
 * (compensated != 0), for given norms (e, f); with e = 0 and f = 1 this is
 * the dot-product itself.  out[0..1] = (Re, Im). */
ORC_EXPORT int orc_dpscl(int64_t m, const double *qr, const double *qi, const double *pr,
                         const double *pi, int eq, double fq, int ep, double fp, int compensated,
                         double *out)
{
  if (m < 1 || !qr || !pr || !out || (!qi) != (!pi)) return ORC_E_ARG;
  if (compensated)
    zdpscl_comp(m, qr, qi, pr, pi, eq, fq, ep, fp, &out[0], &out[1]);
  else
    zdpscl(m, qr, qi, pr, pi, eq, fq, ep, fp, &out[0], &out[1]);
  return ORC_OK;
}

/* Alg. Gram: the non-overflowing scaled Grammian A'' from a21' and the
 * (e,f) norms of g_p (1) and g_q (2). */
static void gram(double a21r, double a21i, int e1, double f1, int e2, double f2, double *a11,
                 double *a22, double *b21r, double *b21i)
{
  double f12 = f1 / f2, f21 = f2 / f1;
  int e12 = e1 - e2, e21 = e2 - e1;
  e12 += flg(f12);
  f12 = ldexp(f12, -flg(f12));
  e21 += flg(f21);
  f21 = ldexp(f21, -flg(f21));
  const int emax = (e12 > e21) ? e12 : e21;
  const int sA = imin((DBL_MAX_EXP - 1) - emax, 0);
  e12 += sA;
  e21 += sA;
  *a11 = ldexp(f12, e12);
  *a22 = ldexp(MUT(15, f21, f12), e21);
  *b21r = ldexp(a21r, sA);
  *b21i = ldexp(a21i, sA);
}

/* Eq. "e:transf" / Alg. zjrot: [x_p x_q] <- [x_p x_q] U P, rows 0..l-1.
 * Real if xpi == NULL (then S is ignored).  Returns the max-norm of the
 * transformed pair (max of |Re| and |Im| parts). */
static double zjrot(int64_t l, double *xpr, double *xpi, double *xqr, double *xqi, double c,
                    double C, double S, int swap)
{
  double M = 0.0;
  for (int64_t i = 0; i < l; ++i) {
    double npr, npi = 0.0, nqr, nqi = 0.0;
    if (xpi) {
      const double pr = xpr[i], pi = xpi[i], qr = xqr[i], qi = xqi[i];
      /* fma(x_q, e', x_p) c, e' = C + iS, complex fma of Eq. "e:zfma" */
      npr = fma(qr, C, fma(-qi, S, pr)) * c;
      npi = fma(qr, S, fma(qi, C, pi)) * c;
      /* fma(x_p, -conj(e'), x_q) c, -conj(e') = -C + iS */
      nqr = fma(pr, -C, fma(-pi, S, qr)) * c;
      nqi = fma(pr, S, fma(pi, -C, qi)) * c;
    } else {
      const double pr = xpr[i], qr = xqr[i];
      npr = fma(qr, C, pr) * c;
      nqr = fma(pr, MUT(7, -C, C), qr) * c;
    }
    M = fmax(M, fmax(fabs(npr), fabs(nqr)));
    if (xpi) M = fmax(M, fmax(fabs(npi), fabs(nqi)));
    if (swap) {
      xpr[i] = nqr;
      xqr[i] = npr;
      if (xpi) {
        xpi[i] = nqi;
        xqi[i] = npi;
      }
    } else {
      xpr[i] = npr;
      xqr[i] = nqr;
      if (xpi) {
        xpi[i] = npi;
        xqi[i] = nqi;
      }
    }
  }
  return M;
}

/* Eq. "e:GScond" in (e, f) form: ||x|| > 2^eta^ upsilon ||y||, eta^ =
 * DBL_MAX_EXP - 1, for ||x|| = 2^ex fx, ||y|| = 2^ey fy. */
static int gs_cond(int ex, double fx, int ey, double fy, double ups)
{
  const int d = ex - ey - (DBL_MAX_EXP - 1);
  const int dc = (d > 4000) ? 4000 : (d < -4000) ? -4000 : d;
  return ldexp(fx / fy, dc) > ups;
}

/* Eq. "e:GS" (Alg. ZGS / DGS): y <- (y / 2^ey - psi x / 2^ex) 2^ey on rows
 * 0..l-1, psi = (psr, psi_i), in the operation order of Alg. ZGS.  Returns
 * the max-norm of the new y. */
static double gsscl(int64_t l, const double *xr, const double *xi, double *yr, double *yi, int ex,
                    int ey, double psr, double psi_i)
{
  double M = 0.0;
  for (int64_t i = 0; i < l; ++i) {
    const double x1 = ldexp(xr[i], -ex), y1 = ldexp(yr[i], -ey);
    if (xi) {
      const double x2 = ldexp(xi[i], -ex), y2 = ldexp(yi[i], -ey);
      const double re = fma(-psr, x1, fma(psi_i, x2, y1));
      const double im = fma(-psr, x2, fma(-psi_i, x1, y2));
      yr[i] = ldexp(re, ey);
      yi[i] = ldexp(im, ey);
      M = fmax(M, fmax(fabs(yr[i]), fabs(yi[i])));
    } else {
      yr[i] = ldexp(fma(MUT(11, -psr, psr), x1, y1), ey);
      M = fmax(M, fabs(yr[i]));
    }
  }
  return M;
}

static void swap_cols(int64_t l, double *a, double *b)
{
  for (int64_t i = 0; i < l; ++i) {
    const double t = a[i];
    a[i] = b[i];
    b[i] = t;
  }
}

/* max-norm of a plane (NaN -> inf), section 3.2 */
static double maxnorm(int64_t m, int64_t n, const double *x, int64_t ld)
{
  double M = 0.0;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) M = fmax(M, fmin(fabs(x[i + j * ld]), INFINITY));
  return M;
}

/* Number of OpenMP threads a parallel region of the oracle uses. */
ORC_EXPORT int orc_num_threads(void)
{
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}


/*
 * orc_vjsvd: Alg. zvjsvd (complex, Gi != NULL) or its real variant dvjsvd.
 *   G (Gr, Gi): m x n, column-major, leading dimension ld, m >= n >= 1;
 *     overwritten by U (columns of unit norm, zero columns stay zero).
 *   V (Vr, Vi): n x n, leading dimension n, overwritten by V.
 *   sig, sig_e, sig_f: n singular values, as doubles and as (e, f).
 *   out_info[5] = {status, sweeps, rotations (low 31 bits), rescales,
 *     Gram-Schmidt transformations (low 31 bits)}.
 *   rotations64 receives the 64-bit rotation count (may be NULL).
 *   permute != 0 applies the column swap P during the sweeps.
 *   compensated != 0 forms the scaled dot-products by Alg. zdpscl' /
 *     ddpscl' (supplement SM2.2) instead of Alg. zdpscl.
 *   skr_shift >= 0 lowers the threshold of the per-step rescaling test of
 *     section 3.2 by 2^skr_shift: step k downscales G (by 2^{s_[k]}, Eq.
 *     "e:skn") when s_(k) - skr_shift < 0 (Eq. "e:skr").  0 is the paper's
 *     test, which the initial scaling keeps from firing unless the max-norm
 *     grows by about 2m; a positive shift makes the branch run on ordinary
 *     inputs, so that the tests can pin it.  Power-of-two scaling is exact,
 *     so without underflow the results do not depend on the shift.
 *   max_steps > 0 stops the sweeps after that many parallel steps (status
 *     not converged), so that a run can be timed on a bounded sample of a
 *     large problem; <= 0: no limit.
 * nthreads <= 0 leaves the OpenMP default.
 */
ORC_EXPORT int orc_vjsvd(int64_t m, int64_t n, double *Gr, double *Gi, int64_t ld, double *Vr,
                         double *Vi, double *sig, double *sig_e, double *sig_f, int max_sweeps,
                         int permute, int compensated, int skr_shift, int64_t max_steps,
                         int nthreads, int32_t *out_info, int64_t *rotations64)
{
  if (m < 1 || n < 1 || m < n || ld < m || max_sweeps < 1 || skr_shift < 0) return ORC_E_ARG;
#ifdef _OPENMP
  /* a num_threads clause, not omp_set_num_threads: later calls keep the
   * default */
  const int n_thr = (nthreads > 0) ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  const int cplx = (Gi != NULL);
  /* V_1 = I */
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      Vr[i + j * n] = (i == j) ? 1.0 : 0.0;
      if (cplx) Vi[i + j * n] = 0.0;
    }
  /* section 3.2, step 1: M~_0 and s_0 = s_[0] (Eq. "e:skn") */
  double Mt = maxnorm(m, n, Gr, ld);
  if (cplx) Mt = fmax(Mt, maxnorm(m, n, Gi, ld));
  if (!(Mt < INFINITY)) return ORC_E_NONFINITE;
  int64_t rotations = 0, gs_count = 0;
  int rescales = 0, sweeps = 0, status = ORC_OK;
  int s = 0;
  /* floor(lg(nu/(varsigma m))) and friends, Eq. "e:skn" / "e:skr" */
  const int lg_skn = cplx ? flg(DBL_MAX / (4.0 * (double)m) / M_SQRT2) : flg(DBL_MAX / (2.0 * (double)m));
  const int lg_skr = cplx ? flg(DBL_MAX / 4.0 / M_SQRT2) : flg(DBL_MAX / 2.0);
  int32_t *tab = NULL;
  int nt = (int)(n + (n & 1));
  if (Mt > 0.0) {
    s = lg_skn - flg(Mt) - 1;
    for (int64_t j = 0; j < n; ++j)
      for (int64_t i = 0; i < m; ++i) {
        Gr[i + j * ld] = ldexp(Gr[i + j * ld], s);
        if (cplx) Gi[i + j * ld] = ldexp(Gi[i + j * ld], s);
      }
    Mt = ldexp(Mt, s);
    tab = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(nt - 1 > 0 ? nt - 1 : 1) * (size_t)(nt / 2 > 0 ? nt / 2 : 1));
    if (!tab) return ORC_E_ARG;
    if (nt >= 2) (void)orc_pairs((int)n, tab);
    /* Eq. "e:tol": upsilon = fl(eps sqrt(m)), eps = 2^-53 */
    const double ups = ldexp(sqrt((double)m), -53);
    const int K = nt - 1, L = nt / 2;
    int converged = (nt < 2);
    int64_t steps_done = 0;
    int stopped = 0;
    for (int C = 0; C < max_sweeps && !converged && !stopped; ++C) {
      int64_t T = 0;
      for (int k = 0; k < K; ++k) {
        if (max_steps > 0 && steps_done == max_steps) {
          stopped = 1;
          break;
        }
        ++steps_done;
        /* steps 2-4 of the heuristic: s_(k) < 0 (Eq. "e:skr") => G is
         * downscaled by 2^{s_[k]} (Eq. "e:skn"), M~ with it, and s_[k] is
         * added to the running scale exponent s */
        const int sk_r = lg_skr - flg(Mt) - (cplx ? 1 : 0);
        if (sk_r - skr_shift < 0) {
          const int sk_n = lg_skn - flg(Mt) - 1;
          for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i < m; ++i) {
              Gr[i + j * ld] = ldexp(Gr[i + j * ld], MUT(19, sk_n, -sk_n));
              if (cplx) Gi[i + j * ld] = ldexp(Gi[i + j * ld], MUT(19, sk_n, -sk_n));
            }
          Mt = ldexp(Mt, sk_n);
          s += MUT(18, sk_n, 0);
          ++rescales;
        }
        int64_t t = 0;
        double Mstep = 0.0;
#pragma omp parallel for schedule(static) num_threads(n_thr) reduction(+ : t, gs_count) \
    reduction(max : Mstep)
        for (int l = 0; l < L; ++l) {
          const int p = tab[2 * ((int64_t)k * L + l)], q = tab[2 * ((int64_t)k * L + l) + 1];
          if (q >= n) continue; /* phantom column */
          double *gpr = Gr + p * ld, *gqr = Gr + q * ld;
          double *gpi = cplx ? Gi + p * ld : NULL, *gqi = cplx ? Gi + q * ld : NULL;
          double *vpr = Vr + p * n, *vqr = Vr + q * n;
          double *vpi = cplx ? Vi + p * n : NULL, *vqi = cplx ? Vi + q * n : NULL;
          int ep, eq;
          double fp, fq;
          colnorm(m, gpr, gpi, &ep, &fp);
          colnorm(m, gqr, gqi, &eq, &fq);
          if (ep == INT_MIN || eq == INT_MIN) {
            if (permute && ef_less(ep, fp, eq, fq)) {
              swap_cols(m, gpr, gqr);
              swap_cols(n, vpr, vqr);
              if (cplx) {
                swap_cols(m, gpi, gqi);
                swap_cols(n, vpi, vqi);
              }
            }
            continue;
          }
          double zr, zi;
          if (compensated)
            zdpscl_comp(m, gqr, gqi, gpr, gpi, eq, fq, ep, fp, &zr, &zi);
          else
            zdpscl(m, gqr, gqi, gpr, gpi, eq, fq, ep, fp, &zr, &zi);
          /* Alg. cvg */
          const double az = cplx ? hypot_naive(zr, zi) : fabs(zr);
          const int rot = (ups <= az);
          /* Alg. Gram, then the EVD (Alg. zbjac2 / dbjac2) */
          double b11, b22, b21r, b21i;
          gram(zr, zi, ep, fp, eq, fq, &b11, &b22, &b21r, &b21i);
          struct evd2 ev;
          if (cplx)
            evd2_complex(b11, b22, b21r, b21i, &ev);
          else
            evd2_real(b11, b22, b21r, &ev);
          const double c = ev.cos_phi, Ct = ev.eatan_re, St = ev.eatan_im;
          const int pbit = permute ? ev.p : 0;
          /* Alg. zvjsvd: when Eq. "e:GScond" holds, Alg. ZGS / DGS replaces
           * zjrot on G; V still takes the rotation */
          const int gs_pq = rot && gs_cond(ep, fp, eq, fq, ups);
          const int gs_qp = rot && !gs_pq && gs_cond(eq, fq, ep, fp, ups);
          if (rot && (gs_pq || gs_qp)) {
            double Mp;
            if (gs_pq) /* g_q against g_p, psi = conj(a21') fq / fp */
              Mp = gsscl(m, gpr, gpi, gqr, gqi, ep, eq, zr * (fq / fp), -(zi * (fq / fp)));
            else /* g_p against g_q, psi = a21' fp / fq */
              Mp = gsscl(m, gqr, gqi, gpr, gpi, eq, ep, zr * (fp / fq), zi * (fp / fq));
            Mp = fmax(Mp, maxnorm(m, 1, gs_pq ? gpr : gqr, ld));
            if (cplx) Mp = fmax(Mp, maxnorm(m, 1, gs_pq ? gpi : gqi, ld));
            if (pbit) {
              swap_cols(m, gpr, gqr);
              if (cplx) swap_cols(m, gpi, gqi);
            }
            (void)zjrot(n, vpr, vpi, vqr, vqi, c, Ct, St, pbit);
            Mstep = fmax(Mstep, Mp);
            ++t;
            ++gs_count;
          } else if (rot) {
            const double Mp = zjrot(m, gpr, gpi, gqr, gqi, c, Ct, St, pbit);
            (void)zjrot(n, vpr, vpi, vqr, vqi, c, Ct, St, pbit);
            Mstep = fmax(Mstep, Mp);
            ++t;
          } else if (pbit) {
            swap_cols(m, gpr, gqr);
            swap_cols(n, vpr, vqr);
            if (cplx) {
              swap_cols(m, gpi, gqi);
              swap_cols(n, vpi, vqi);
            }
          }
        }
        T += t;
        Mt = fmax(Mt, Mstep);
      }
      rotations += T;
      sweeps = C + 1;
      if (T == 0 && !stopped) converged = 1;
    }
    if (!converged) status = ORC_NOT_CONVERGED;
  }
  /* section 4.2.1: U = G columns scaled by 2^-e_j and divided by f_j;
   * sigma_j = (e_j - s, f_j) */
  int *ee = (int *)malloc(sizeof(int) * (size_t)n);
  double *ff = (double *)malloc(sizeof(double) * (size_t)n);
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!ee || !ff || !perm) {
    free(tab); free(ee); free(ff); free(perm);
    return ORC_E_ARG;
  }
  for (int64_t j = 0; j < n; ++j) {
    colnorm(m, Gr + j * ld, cplx ? Gi + j * ld : NULL, &ee[j], &ff[j]);
    if (ee[j] == INT_MIN) {
      for (int64_t i = 0; i < m; ++i) {
        Gr[i + j * ld] = 0.0;
        if (cplx) Gi[i + j * ld] = 0.0;
      }
      continue;
    }
    for (int64_t i = 0; i < m; ++i) {
      Gr[i + j * ld] = ldexp(Gr[i + j * ld], -ee[j]) / ff[j];
      if (cplx) Gi[i + j * ld] = ldexp(Gi[i + j * ld], -ee[j]) / ff[j];
    }
    ee[j] -= s;
  }
  /* stable sort by sigma, non-increasing (insertion sort: n is small here) */
  for (int64_t j = 0; j < n; ++j) perm[j] = j;
  for (int64_t j = 1; j < n; ++j) {
    const int64_t x = perm[j];
    int64_t i = j - 1;
    while (i >= 0) {
      const int64_t y = perm[i];
      /* y goes after x iff sigma_y < sigma_x (zero norms are smallest) */
      const int y_zero = (ee[y] == INT_MIN), x_zero = (ee[x] == INT_MIN);
      int y_less;
      if (y_zero || x_zero) y_less = y_zero && !x_zero;
      else y_less = ef_less(ee[y], ff[y], ee[x], ff[x]);
      if (!y_less) break;
      perm[i + 1] = y;
      --i;
    }
    perm[i + 1] = x;
  }
  double *tmp = (double *)malloc(sizeof(double) * (size_t)(m > n ? m : n) * (size_t)n);
  if (!tmp) {
    free(tab); free(ee); free(ff); free(perm);
    return ORC_E_ARG;
  }
  for (int plane = 0; plane < (cplx ? 2 : 1); ++plane) {
    double *Gx = plane ? Gi : Gr, *Vx = plane ? Vi : Vr;
    for (int64_t j = 0; j < n; ++j) memcpy(tmp + j * m, Gx + perm[j] * ld, sizeof(double) * (size_t)m);
    for (int64_t j = 0; j < n; ++j) memcpy(Gx + j * ld, tmp + j * m, sizeof(double) * (size_t)m);
    for (int64_t j = 0; j < n; ++j) memcpy(tmp + j * n, Vx + perm[j] * n, sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) memcpy(Vx + j * n, tmp + j * n, sizeof(double) * (size_t)n);
  }
  for (int64_t j = 0; j < n; ++j) {
    const int64_t y = perm[j];
    const int zero = (ee[y] == INT_MIN);
    if (sig) sig[j] = zero ? 0.0 : ldexp(ff[y], ee[y]);
    if (sig_e) sig_e[j] = zero ? -INFINITY : (double)ee[y];
    if (sig_f) sig_f[j] = zero ? 1.0 : ff[y];
  }
  free(tmp);
  free(tab);
  free(ee);
  free(ff);
  free(perm);
  if (out_info) {
    out_info[0] = status;
    out_info[1] = sweeps;
    out_info[2] = (int32_t)(rotations & 0x7fffffff);
    out_info[3] = rescales;
    out_info[4] = (int32_t)(gs_count & 0x7fffffff);
  }
  if (rotations64) *rotations64 = rotations;
  return status;
}

/* ------------------------------------------------------------------------
 * Thin real SVD adjoint (Townsend 2016, "Differentiating the singular value
 * decomposition"; Ionescu, Vantzos, Sminchisescu 2015):
 *   Abar = U [ (F o (U^T Ubar - Ubar^T U)) S + diag(Sbar)
 *              + S (F o (V^T Vbar - Vbar^T V)) ] V^T
 *        + (I - U U^T) Ubar S^-1 V^T,
 *   F_ij = 1/(s_j^2 - s_i^2) for i != j, F_ii = 0.
 * U, Ubar, Abar: m x n; V, Vbar: n x n; all column-major, leading dimension
 * m or n.  Vbar may be NULL (zero).  Plain triple loops. */
ORC_EXPORT int orc_svd_adjoint(int64_t m, int64_t n, const double *U, const double *s,
                               const double *V, const double *Ubar, const double *sbar,
                               const double *Vbar, double *Abar)
{
  double *J = (double *)calloc((size_t)(n * n), sizeof(double));
  double *Kv = (double *)calloc((size_t)(n * n), sizeof(double));
  double *In = (double *)calloc((size_t)(n * n), sizeof(double));
  double *W = (double *)calloc((size_t)(m * n), sizeof(double));
  if (!J || !Kv || !In || !W) {
    free(J); free(Kv); free(In); free(W);
    return ORC_E_ARG;
  }
  /* J = U^T Ubar, Kv = V^T Vbar */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int64_t r = 0; r < m; ++r) acc += U[r + i * m] * Ubar[r + j * m];
      J[i + j * n] = acc;
      double acc2 = 0.0;
      if (Vbar)
        for (int64_t r = 0; r < n; ++r) acc2 += V[r + i * n] * Vbar[r + j * n];
      Kv[i + j * n] = acc2;
    }
  /* inner = (F o (J - J^T)) S + diag(sbar) + S (F o (Kv - Kv^T)) */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double v = 0.0;
      if (i != j) {
        const double F = MUT(12, 1.0 / (s[j] * s[j] - s[i] * s[i]), 1.0 / (s[i] * s[i] - s[j] * s[j]));
        v = F * (J[i + j * n] - J[j + i * n]) * s[j] + s[i] * F * (Kv[i + j * n] - Kv[j + i * n]);
      } else {
        v = sbar ? sbar[i] : 0.0;
      }
      In[i + j * n] = v;
    }
  /* W = U inner + (Ubar - U J) diag(1/s) */
  for (int64_t r = 0; r < m; ++r)
    for (int64_t j = 0; j < n; ++j) {
      double a = 0.0, uj = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        a += U[r + i * m] * In[i + j * n];
        uj += U[r + i * m] * J[i + j * n];
      }
      W[r + j * m] = a + (Ubar[r + j * m] - uj) / s[j];
    }
  /* Abar = W V^T */
  for (int64_t r = 0; r < m; ++r)
    for (int64_t c = 0; c < n; ++c) {
      double acc = 0.0;
      for (int64_t j = 0; j < n; ++j) acc += W[r + j * m] * V[c + j * n];
      Abar[r + c * m] = acc;
    }
  free(J);
  free(Kv);
  free(In);
  free(W);
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Batches for the timings of the batched workloads: the matrices are
 * independent, so the OpenMP threads share them out (dynamic schedule),
 * each matrix's SVD running on one thread.  Nothing here changes what one
 * SVD or one adjoint computes. */

/* Real SVDs of count matrices packed column-major back to back: matrix i
 * (m[i] x n[i], leading dimension m[i]) at G + offA[i], overwritten by U;
 * V_i (n[i] x n[i]) at V + offV[i]; sigma_i at sig + offS[i].  status[i]
 * receives orc_vjsvd's return value.  nthreads <= 0: the OpenMP default. */
ORC_EXPORT int orc_vjsvd_batch(int64_t count, const int64_t *m, const int64_t *n,
                               const int64_t *offA, const int64_t *offV, const int64_t *offS,
                               double *G, double *V, double *sig, int max_sweeps, int nthreads,
                               int32_t *status)
{
  if (count < 0 || !m || !n || !offA || !offV || !offS || !G || !V || !sig || !status)
    return ORC_E_ARG;
#ifdef _OPENMP
  const int nt = (nthreads > 0) ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int64_t i = 0; i < count; ++i)
    status[i] = orc_vjsvd(m[i], n[i], G + offA[i], NULL, m[i], V + offV[i], NULL, sig + offS[i],
                          NULL, NULL, max_sweeps, 0, 0, 0, 0, 1, NULL, NULL);
  return ORC_OK;
}

/* orc_svd_adjoint for count matrices of one shape m x n packed back to
 * back (U, Ubar, Abar: m n each; V: n n; s, sbar: n); Vbar is zero. */
ORC_EXPORT int orc_svd_adjoint_batch(int64_t count, int64_t m, int64_t n, const double *U,
                                     const double *s, const double *V, const double *Ubar,
                                     const double *sbar, double *Abar, int nthreads)
{
  if (count < 0 || m < 1 || n < 1) return ORC_E_ARG;
  int bad = 0;
#ifdef _OPENMP
  const int nt = (nthreads > 0) ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt) reduction(| : bad)
#endif
  for (int64_t i = 0; i < count; ++i)
    bad |= (orc_svd_adjoint(m, n, U + i * m * n, s + i * n, V + i * n * n, Ubar + i * m * n,
                            sbar + i * n, NULL, Abar + i * m * n) != ORC_OK);
  return bad ? ORC_E_ARG : ORC_OK;
}

/* The OpenMP environment in force for the oracle's parallel loops:
 * out[0] = threads a parallel region gets, out[1] = omp_get_proc_bind()
 * (0 false, 1 true, 2 primary, 3 close, 4 spread), out[2] = number of
 * places, out[3] = omp_get_dynamic().  Without OpenMP: {1, 0, 0, 0}. */
ORC_EXPORT void orc_omp_state(int32_t *out)
{
#ifdef _OPENMP
  out[0] = omp_get_max_threads();
  out[1] = (int32_t)omp_get_proc_bind();
  out[2] = omp_get_num_places();
  out[3] = omp_get_dynamic();
#else
  out[0] = 1;
  out[1] = out[2] = out[3] = 0;
#endif
}

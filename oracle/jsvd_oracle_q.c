/*
 * jsvd_oracle_q.c -- the binary128 twin of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see jsvd_oracle.c).  The same methods as the
 * FP64 oracle in IEEE binary128 (_Float128 with glibc's f128 functions), so
 * that the tests can measure the FP64 oracle against results carrying 60
 * more bits:
 *   orc_q_zsjac2  the 2x2 Hermitian EVD of section 2 (the equations the
 *                 FP64 oracle restates) with the binary128 constants the
 *                 paper prescribes for other formats (section 2.4: nu =
 *                 FLT128_MAX, fl(sqrt nu), mu = FLT128_TRUE_MIN, eta =
 *                 floor(lg(nu/8)) = FLT128_MAX_EXP - 4);
 *   orc_q_vjsvd   the one-sided Jacobi SVD of Alg. zvjsvd: the same
 *                 round-robin ordering, the scaled dot-products of Alg.
 *                 zdpscl, the test of Eq. "e:tol" with eps = 2^-113, the
 *                 scaled Grammian of Alg. Gram and its EVD above, the
 *                 transformations of Eq. "e:transf", the final sort.  The
 *                 binary128 range holds every square and product of binary64
 *                 data, so the scalings of section 3.2 and the (e, f) norms
 *                 are not needed: norms are plain square roots of sums.
 * Outputs are returned as pairs of doubles (hi, lo) with hi + lo the
 * binary128 value to about 2^-106 relative, or rounded to double where the
 * tests need no more.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* Mutation points for the pin tests (see jsvd_oracle.c): -DORC_MUTANT=k
 * plants mistake k; by default the plain twin. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif
#define MUT(k, good, bad) ((ORC_MUTANT == (k)) ? (bad) : (good))

typedef _Float128 q;

/* from jsvd_oracle.c: the round-robin ordering table */
int orc_pairs(int n, int32_t *tab);

static void split(q x, double *hi, double *lo)
{
  const double h = (double)x;
  *hi = h;
  *lo = (double)(x - (q)h);
}

/* floor(lg x) for finite x > 0. */
static int flg_q(q x)
{
  int e;
  (void)frexpf128(x, &e);
  return e - 1;
}

static int imin_q(int a, int b) { return a <= b ? a : b; }

/* zeta_x of Eq. "e:z" with the binary128 constants of section 2.4:
 * eta - floor(lg max(|x|, mu-check)), eta = floor(lg(nu/8)), nu =
 * FLT128_MAX, mu-check = FLT128_TRUE_MIN. */
static int zeta_elem_q(q x)
{
  const int eta = flg_q(FLT128_MAX / 8);
  return eta - flg_q(fmaxf128(fabsf128(x), FLT128_TRUE_MIN));
}

/* Alg. hypot in binary128 (Eq. "e:hypot"). */
static q hypot_naive_q(q x, q y)
{
  const q ax = fabsf128(x), ay = fabsf128(y);
  const q m = fminf128(ax, ay), M = fmaxf128(ax, ay);
  const q ratio = fmaxf128(m / M, 0);
  return sqrtf128(fmaf128(ratio, ratio, 1)) * M;
}

/* The EVD of section 2 in binary128: the scaling of Eq. "e:z", the polar
 * form of Eq. "e:zpolar", then Eq. "e:tan2", "e:jactan", "e:jacsec" and
 * "e:lamsec".  Returns cos(phi), e^{i alpha} tan(phi), the scaled
 * eigenvalues lambda' and zeta. */
static void zsjac2_q(q a11, q a22, q a21r, q a21i, q *cphi, q *ctr, q *cti, q *l1, q *l2, int *zeta)
{
  const int z = imin_q(imin_q(zeta_elem_q(a11), zeta_elem_q(a22)),
                       imin_q(zeta_elem_q(a21r), zeta_elem_q(a21i)));
  a11 = ldexpf128(a11, z);
  a22 = ldexpf128(a22, z);
  a21r = ldexpf128(a21r, z);
  a21i = ldexpf128(a21i, z);
  /* Eq. "e:zpolar" */
  const q abs_a21 = hypot_naive_q(a21r, a21i);
  const q cos_alpha = copysignf128(fminf128(fabsf128(a21r) / abs_a21, 1), a21r);
  const q sin_alpha = a21i / fmaxf128(abs_a21, FLT128_TRUE_MIN);
  /* Eq. "e:tan2" */
  const q two_abs_a21 = 2 * abs_a21;
  const q a = a11 - a22;
  const q tan_2phi =
      copysignf128(fminf128(fmaxf128(two_abs_a21 / fabsf128(a), 0), sqrtf128(FLT128_MAX)), a);
  /* Eq. "e:jactan" */
  const q t = tan_2phi / (MUT(16, 1, 2) + sqrtf128(fmaf128(tan_2phi, tan_2phi, 1)));
  /* Eq. "e:jacsec" */
  const q sec2 = fmaf128(t, t, 1);
  *cphi = 1 / sqrtf128(sec2);
  *ctr = cos_alpha * t;
  *cti = sin_alpha * t;
  /* Eq. "e:lamsec" */
  *l1 = fmaf128(fmaf128(a22, t, two_abs_a21), t, a11) / sec2;
  *l2 = fmaf128(fmaf128(a11, t, -two_abs_a21), t, a22) / sec2;
  *zeta = z;
}

/* Batched complex (a21i = 0 for a real matrix) EVD in binary128 of double
 * inputs; outputs as (hi, lo) pairs: out[2 i], out[2 i + 1].  lam1, lam2
 * are the backscaled eigenvalues 2^-zeta lambda'. */
ORC_EXPORT void orc_q_zsjac2(int64_t r, const double *a11, const double *a22, const double *a21r,
                             const double *a21i, double *cphi, double *ctr, double *cti,
                             double *lam1, double *lam2)
{
  for (int64_t i = 0; i < r; ++i) {
    q c, tr, ti, l1, l2;
    int z;
    zsjac2_q(a11[i], a22[i], a21r[i], a21i ? a21i[i] : 0.0, &c, &tr, &ti, &l1, &l2, &z);
    split(c, cphi + 2 * i, cphi + 2 * i + 1);
    split(tr, ctr + 2 * i, ctr + 2 * i + 1);
    split(ti, cti + 2 * i, cti + 2 * i + 1);
    split(ldexpf128(l1, -z), lam1 + 2 * i, lam1 + 2 * i + 1);
    split(ldexpf128(l2, -z), lam2 + 2 * i, lam2 + 2 * i + 1);
  }
}

/* ||x|| of a column (one or two planes) */
static q colnorm_q(int64_t m, const q *xr, const q *xi)
{
  q s = 0;
  for (int64_t i = 0; i < m; ++i) {
    s = fmaf128(xr[i], xr[i], s);
    if (xi) s = fmaf128(xi[i], xi[i], s);
  }
  return sqrtf128(s);
}

/* Eq. "e:transf": [x_p x_q] <- [x_p x_q] [[1, -conj(e)], [e, 1]] c */
static void rot_q(int64_t l, q *xpr, q *xpi, q *xqr, q *xqi, q c, q C, q S)
{
  for (int64_t i = 0; i < l; ++i) {
    if (xpi) {
      const q pr = xpr[i], pi = xpi[i], qr = xqr[i], qi = xqi[i];
      xpr[i] = fmaf128(qr, C, fmaf128(-qi, S, pr)) * c;
      xpi[i] = fmaf128(qr, S, fmaf128(qi, C, pi)) * c;
      xqr[i] = fmaf128(pr, -C, fmaf128(-pi, S, qr)) * c;
      xqi[i] = fmaf128(pr, S, fmaf128(pi, -C, qi)) * c;
    } else {
      const q pr = xpr[i], qr = xqr[i];
      xpr[i] = fmaf128(qr, C, pr) * c;
      xqr[i] = fmaf128(pr, -C, qr) * c;
    }
  }
}

/*
 * orc_q_vjsvd: the SVD of the m x n double matrix (Ar, Ai; Ai NULL for
 * real; column-major, leading dimension ld) in binary128.  Outputs: sigma
 * (hi, lo) pairs non-increasing (2 n doubles each array), U (m x n) and V
 * (n x n) rounded to double, column-major (planes for complex), sweeps.
 * Returns 0, or 1 if max_sweeps passed without convergence, -1 on bad
 * arguments.
 */
ORC_EXPORT int orc_q_vjsvd(int64_t m, int64_t n, const double *Ar, const double *Ai, int64_t ld,
                           double *sig_hi, double *sig_lo, double *Ur, double *Ui, double *Vr,
                           double *Vi, int max_sweeps, int32_t *sweeps_out)
{
  if (m < 1 || n < 1 || n > m || ld < m || max_sweeps < 1) return -1;
  const int cplx = (Ai != NULL);
  q *Gr = malloc(sizeof(q) * (size_t)(m * n)), *Gi = cplx ? malloc(sizeof(q) * (size_t)(m * n)) : NULL;
  q *Wr = malloc(sizeof(q) * (size_t)(n * n)), *Wi = cplx ? malloc(sizeof(q) * (size_t)(n * n)) : NULL;
  const int nt = (int)(n + (n & 1));
  int32_t *tab = malloc(sizeof(int32_t) * 2 * (size_t)(nt > 1 ? nt - 1 : 1) * (size_t)(nt / 2 > 0 ? nt / 2 : 1));
  q *nrm = malloc(sizeof(q) * (size_t)n);
  int64_t *perm = malloc(sizeof(int64_t) * (size_t)n);
  if (!Gr || !Wr || !tab || !nrm || !perm || (cplx && (!Gi || !Wi))) {
    free(Gr); free(Gi); free(Wr); free(Wi); free(tab); free(nrm); free(perm);
    return -1;
  }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i) {
      Gr[i + j * m] = Ar[i + j * ld];
      if (cplx) Gi[i + j * m] = Ai[i + j * ld];
    }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      Wr[i + j * n] = (i == j) ? 1 : 0;
      if (cplx) Wi[i + j * n] = 0;
    }
  if (nt >= 2) (void)orc_pairs((int)n, tab);
  const q ups = ldexpf128(sqrtf128((q)m), -113); /* Eq. "e:tol", eps = 2^-113 */
  const int K = nt - 1, L = nt / 2;
  int sweeps = 0, converged = (nt < 2);
  for (int C = 0; C < max_sweeps && !converged; ++C) {
    int64_t T = 0;
    for (int k = 0; k < K; ++k) {
      for (int l = 0; l < L; ++l) {
        const int p = tab[2 * (k * L + l)], qq = tab[2 * (k * L + l) + 1];
        if (qq >= n) continue;
        q *gpr = Gr + p * m, *gqr = Gr + qq * m;
        q *gpi = cplx ? Gi + p * m : NULL, *gqi = cplx ? Gi + qq * m : NULL;
        const q np_ = colnorm_q(m, gpr, gpi), nq_ = colnorm_q(m, gqr, gqi);
        if (np_ == 0 || nq_ == 0) continue;
        /* Alg. zdpscl: g_q^* g_p / (||g_q|| ||g_p||) */
        q zr = 0, zi = 0;
        for (int64_t i = 0; i < m; ++i) {
          zr = fmaf128(gqr[i], gpr[i], zr);
          if (cplx) {
            zi = fmaf128(gqr[i], gpi[i], zi);
            zr = fmaf128(gqi[i], gpi[i], zr);
            zi = fmaf128(-gqi[i], gpr[i], zi);
          }
        }
        const q d = nq_ * np_;
        zr /= d;
        zi /= d;
        q az = fabsf128(zr);
        if (cplx) { /* Alg. hypot */
          const q x = fabsf128(zr), y = fabsf128(zi);
          const q mn = fminf128(x, y), mx = fmaxf128(x, y);
          const q t = fmaxf128(mn / mx, 0);
          az = sqrtf128(fmaf128(t, t, 1)) * mx;
        }
        if (!(ups <= az)) continue;
        ++T;
        /* Alg. Gram (no scaling needed here) and the EVD */
        q c, tr, ti, l1, l2;
        int z;
        zsjac2_q(np_ / nq_, nq_ / np_, zr, zi, &c, &tr, &ti, &l1, &l2, &z);
        rot_q(m, gpr, gpi, gqr, gqi, c, tr, ti);
        rot_q(n, Wr + p * n, cplx ? Wi + p * n : NULL, Wr + qq * n, cplx ? Wi + qq * n : NULL, c,
              tr, ti);
      }
    }
    sweeps = C + 1;
    if (T == 0) converged = 1;
  }
  for (int64_t j = 0; j < n; ++j) {
    nrm[j] = colnorm_q(m, Gr + j * m, cplx ? Gi + j * m : NULL);
    perm[j] = j;
  }
  /* stable sort, non-increasing */
  for (int64_t j = 1; j < n; ++j) {
    const int64_t x = perm[j];
    int64_t i = j - 1;
    while (i >= 0 && nrm[perm[i]] < nrm[x]) {
      perm[i + 1] = perm[i];
      --i;
    }
    perm[i + 1] = x;
  }
  for (int64_t j = 0; j < n; ++j) {
    const int64_t y = perm[j];
    split(nrm[y], sig_hi + j, sig_lo + j);
    for (int64_t i = 0; i < m; ++i) {
      Ur[i + j * m] = nrm[y] == 0 ? 0.0 : (double)(Gr[i + y * m] / nrm[y]);
      if (cplx) Ui[i + j * m] = nrm[y] == 0 ? 0.0 : (double)(Gi[i + y * m] / nrm[y]);
    }
    for (int64_t i = 0; i < n; ++i) {
      Vr[i + j * n] = (double)Wr[i + y * n];
      if (cplx) Vi[i + j * n] = (double)Wi[i + y * n];
    }
  }
  if (sweeps_out) *sweeps_out = sweeps;
  free(Gr); free(Gi); free(Wr); free(Wi); free(tab); free(nrm); free(perm);
  return converged ? 0 : 1;
}

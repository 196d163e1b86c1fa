// Host check of the integer-pipe binary64 division and square root
// (paper_2202_08361_gb300/csrc/fp64soft.cuh, fp64sel.cuh) against the host's
// IEEE arithmetic (SSE2 / AArch64 FP: correctly rounded to nearest even).
// The select-based forms (div_rn_sel, sqrt_rn_sel, ldexp_rn_sel) are
// checked the same way, ldexp_rn_sel and ldexp_rn_uni against the host's
// ldexp, and gt_scaled_pos against the comparison of the host's ldexp
// result (positive normal operands).
// Usage: soft_fp64_check N seed -> prints "div_bad sqrt_bad div_sel_bad
// sqrt_sel_bad ldexp_sel_bad ldexp_uni_bad gt_scaled_pos_bad" and exits 0.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fp64soft.cuh"
#include "fp64sel.cuh"

static uint64_t s_state;
static uint64_t rnd()
{
  // splitmix64
  uint64_t z = (s_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double bitsd(uint64_t u)
{
  double x;
  memcpy(&x, &u, 8);
  return x;
}
static uint64_t dbits(double x)
{
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
}

// finite doubles from several families
static double draw()
{
  const uint64_t r = rnd();
  switch (r & 7) {
    case 0: {  // any finite bit pattern
      uint64_t u;
      do u = rnd(); while (((u >> 52) & 0x7FF) == 0x7FF);
      return bitsd(u);
    }
    case 1:  // subnormal
      return bitsd((rnd() & 0x000FFFFFFFFFFFFFull) | (rnd() & 0x8000000000000000ull));
    case 2:  // moderate exponents
      return ldexp(1.0 + (double)(rnd() >> 11) * 0x1p-53, (int)(rnd() % 200) - 100);
    case 3:  // powers of two and their neighbours
      return nextafter(ldexp(1.0, (int)(rnd() % 2090) - 1074), (rnd() & 1) ? INFINITY : 0.0);
    case 4:  // mantissas with few bits set (exact quotients likely)
      return ldexp((double)((rnd() % 4096) + 1), (int)(rnd() % 100) - 50);
    case 5:  // near the top of the range
      return ldexp(1.0 + (double)(rnd() >> 11) * 0x1p-53, 1000 + (int)(rnd() % 23));
    case 6:  // near the bottom of the normal range
      return ldexp(1.0 + (double)(rnd() >> 11) * 0x1p-53, -1022 + (int)(rnd() % 60));
    default:
      return (double)(rnd() >> 11) * 0x1p-53 + 1.0;
  }
}

int main(int argc, char **argv)
{
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  s_state = argc > 2 ? strtoull(argv[2], nullptr, 10) : 1;
  long bad_div = 0, bad_sqrt = 0, bad_div_sel = 0, bad_sqrt_sel = 0, bad_ldexp_sel = 0;
  long bad_ldexp_uni = 0, bad_gt = 0;
  for (long i = 0; i < n; ++i) {
    double a = draw(), b = draw();
    if (b == 0.0) b = 1.0;
    // also near-ties: a = q b rounded, for q with a 53-bit mantissa
    if ((i & 15) == 0) {
      const double q = ldexp(1.0 + (double)(rnd() >> 11) * 0x1p-53, (int)(rnd() % 40) - 20);
      a = q * b;
      if (!std::isfinite(a) || a == 0.0) a = 1.0;
    }
    const double ref = a / b;
    const double got = jsvd::soft::div_rn(a, b);
    if (dbits(ref) != dbits(jsvd::soft::div_rn_sel(a, b))) ++bad_div_sel;
    if (dbits(ref) != dbits(got)) {
      if (bad_div < 5)
        fprintf(stderr, "div %a / %a: ref %a got %a\n", a, b, ref, got);
      ++bad_div;
    }
    double x = fabs(draw());
    if ((i & 7) == 0) {  // squares and their neighbours
      const double s = fabs(draw());
      x = s * s;
      if (!std::isfinite(x)) x = 2.0;
      if (rnd() & 1) x = nextafter(x, (rnd() & 1) ? INFINITY : 0.0);
    }
    const double rs = sqrt(x);
    const double gs = jsvd::soft::sqrt_rn(x);
    if (dbits(rs) != dbits(jsvd::soft::sqrt_rn_sel(x))) ++bad_sqrt_sel;
    // x 2^k over the whole range, subnormal results (rounded) included
    const int k = (int)(rnd() % 4200) - 2100;
    const double y = draw();
    if (dbits(ldexp(y, k)) != dbits(jsvd::soft::ldexp_rn_sel(y, k))) {
      if (bad_ldexp_sel < 5) fprintf(stderr, "ldexp %a %d: ref %a got %a\n", y, k, ldexp(y, k), jsvd::soft::ldexp_rn_sel(y, k));
      ++bad_ldexp_sel;
    }
    if (dbits(ldexp(y, k)) != dbits(jsvd::soft::ldexp_rn_uni(y, k))) ++bad_ldexp_uni;
    // fl(q 2^d) > u on bit patterns, q and u positive normal; u also just
    // above, just below or equal to q 2^d
    {
      auto pos_normal = [&]() {
        double v = fabs(draw());
        return (v >= 0x1p-1022) ? v : ldexp(1.0 + (double)(rnd() >> 11) * 0x1p-53, (int)(rnd() % 2046) - 1022);
      };
      const double q = pos_normal();
      const int d = (int)(rnd() % 8001) - 4000;
      double u = pos_normal();
      if ((i & 3) == 0) {
        const double t = ldexp(q, d);
        const double at = fabs(t);
        const uint64_t pick = rnd() % 3;  // just above, just below, equal
        const double c = pick == 2 ? at : nextafter(at, pick ? INFINITY : 0.0);
        if (c >= 0x1p-1022 && c <= DBL_MAX) u = c;
      }
      if ((dbits(ldexp(q, d)) > dbits(u)) != jsvd::soft::gt_scaled_pos(q, d, u)) ++bad_gt;
    }
    if (dbits(rs) != dbits(gs)) {
      if (bad_sqrt < 5) fprintf(stderr, "sqrt %a: ref %a got %a\n", x, rs, gs);
      ++bad_sqrt;
    }
  }
  printf("%ld %ld %ld %ld %ld %ld %ld\n", bad_div, bad_sqrt, bad_div_sel, bad_sqrt_sel,
         bad_ldexp_sel, bad_ldexp_uni, bad_gt);
  return 0;
}

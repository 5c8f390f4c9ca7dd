/* The shared-reciprocal division of the interpolation kernels, restated on
 * the host: y = RN(1/b); q0 = RN(a y); q1 = RN(q0 + RN(a - b q0) y);
 * q2 = RN(q1 + (a - b q1) y), which Markstein's theorem makes RN(a/b) when
 * q1 is within one ulp of a/b and no quantity leaves the normal range. The
 * test compares q2 with a / b bit for bit on generated pairs whose binary
 * exponents lie in [-400, 400] (the range the kernels take this path for).
 * fma() from the C library is the correctly rounded fused multiply-add. */
#include <math.h>
#include <stdint.h>
#include <string.h>

static uint64_t mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static double make(uint64_t r, int kind, int e) {
  uint64_t m = r & 0xfffffffffffffULL;
  if (kind == 1) m = r & 0xffULL;                        /* mantissa near 1 */
  if (kind == 2) m = 0xfffffffffffffULL - (r & 0xffULL); /* near 2 */
  if (kind == 3) m = (r & 0xfffffffULL) << 24;           /* short mantissa */
  uint64_t bits = (r >> 63) << 63 | (uint64_t)(1023 + e) << 52 | m;
  double x;
  memcpy(&x, &bits, sizeof x);
  return x;
}

double shared_reciprocal_quotient(double a, double b, double y) {
  double q = a * y;
  double r = fma(-q, b, a);
  q = fma(r, y, q);
  r = fma(-q, b, a);
  return fma(r, y, q);
}

/* the planted mistake: the product with the reciprocal, uncorrected */
double uncorrected_quotient(double a, double b, double y) {
  (void)b;
  return a * y;
}

/* mismatches among n pairs from seed (corrected: the kernels' sequence, else
 * the planted one); the first one's operands in first[0..1] */
long long count_mismatches(long long n, uint64_t seed, int corrected, double* first) {
  long long bad = 0;
  for (long long i = 0; i < n; ++i) {
    uint64_t r1 = mix(seed ^ (uint64_t)(2 * i)), r2 = mix(seed ^ (uint64_t)(2 * i + 1));
    uint64_t r3 = mix(r1 ^ r2);
    int ka = (int)(r3 & 3), kb = (int)((r3 >> 2) & 3);
    int ea = (int)((r3 >> 8) % 801) - 400, eb = (int)((r3 >> 20) % 801) - 400;
    if ((r3 >> 40) & 1) {
      ea = (int)((r3 >> 8) % 9) - 4;
      eb = (int)((r3 >> 20) % 9) - 4;
    }
    double a = make(r1, ka, ea), b = make(r2, kb, eb);
    double y = 1.0 / b;
    double q = corrected ? shared_reciprocal_quotient(a, b, y) : uncorrected_quotient(a, b, y);
    double d = a / b;
    if (memcmp(&q, &d, sizeof q) != 0) {
      if (bad == 0) {
        first[0] = a;
        first[1] = b;
      }
      ++bad;
    }
  }
  return bad;
}

/* Host check of the method the device kick uses for its divisions by the
 * pair mass M (Eqs. 12-13): q0 = x y with y the correctly rounded 1/M,
 * Markstein's correction q = q0 + (x - M q0) y, then the remainder check
 * that keeps q only when |x - M q| < M s/2 (s: the spacing of the doubles
 * next to q on the side of x/M).  The same steps and bit operations as the
 * device, in C with the C library's correctly rounded fma().
 *
 * Counts, over seeded random cases (significands uniform, near 1, near 2
 * and near powers of two; exponents within +-500; both signs):
 *   wrong    - results (kept q, else the division) that differ from x / M
 *   fallback - cases where the check rejected q
 *   kept_bad - wrong quotients (the neighbours 1 and 2 ulp away from x / M)
 *              that the check kept
 *   lost     - correctly rounded quotients that the check rejected
 * Usage: kick_division_check N SEED; prints the four counts. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t state;
static uint64_t next_u64(void) { /* xorshift64 */
  state ^= state << 13;
  state ^= state >> 7;
  state ^= state << 17;
  return state;
}
static uint64_t bits(double d) { uint64_t b; memcpy(&b, &d, 8); return b; }
static double from_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }

static int in_range(double v, int positive) {
  const uint64_t b = bits(v);
  const unsigned e = positive ? (unsigned)(b >> 52) : (unsigned)(b >> 52) & 0x7FFu;
  return e - 523u < 1000u;
}

static int keep(double x, double M, double q) {
  const double r = fma(-M, q, x);
  const uint64_t qb = bits(q), rb = bits(r);
  const int toward0 = ((qb ^ rb) >> 63) != 0;
  const int pow2 = (qb & 0xFFFFFFFFFFFFFull) == 0;
  const long long k = (long long)((qb >> 52) & 0x7FFu) - 1076 - ((toward0 && pow2) ? 1 : 0);
  const uint64_t half_gap = bits(M) + ((uint64_t)k << 52);
  return (rb & 0x7FFFFFFFFFFFFFFFull) < half_gap;
}

static double make(int e, uint64_t sig, int neg) {
  return from_bits(((uint64_t)neg << 63) | ((uint64_t)(1023 + e) << 52) |
                   (sig & 0xFFFFFFFFFFFFFull));
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  state = argc > 2 ? strtoull(argv[2], 0, 10) * 0x9E3779B97F4A7C15ull + 1 : 1;
  long wrong = 0, fallback = 0, kept_bad = 0, lost = 0;
  for (long i = 0; i < n; ++i) {
    const uint64_t r = next_u64();
    uint64_t sm = next_u64(), sx = next_u64();
    switch (i % 5) {
      case 1: sm |= 0xFFFFFF0000000ull; break;                              /* M near 2 */
      case 2: sm |= 0xFFFFFF0000000ull; sx |= 0xFFFFFF0000000ull; break;    /* both */
      case 3: sm &= 0x00000FFFFFFFFull; break;                              /* M near 1 */
      case 4: sx &= 0xFull; break;                                          /* x near 2^k */
    }
    int em = (int)(r % 1001) - 500, ex = (int)((r >> 10) % 1001) - 500;
    if (i % 3 == 0) { em = (int)(r % 9) - 4; ex = (int)((r >> 10) % 9) - 4; }
    const double M = make(em, sm, 0), x = make(ex, sx, (int)((r >> 20) & 1));
    if (!(in_range(M, 1) && in_range(x, 0))) continue;
    const double y = 1.0 / M;
    const double q0 = x * y;
    const double q = fma(fma(-M, q0, x), y, q0);
    const double t = x / M;
    double res = t;
    if (keep(x, M, q)) res = q; else ++fallback;
    if (bits(res) != bits(t)) ++wrong;
    const double up = nextafter(t, INFINITY), dn = nextafter(t, -INFINITY);
    const double cand[4] = {up, dn, nextafter(up, INFINITY), nextafter(dn, -INFINITY)};
    for (int c = 0; c < 4; ++c) kept_bad += keep(x, M, cand[c]);
    lost += !keep(x, M, t);
  }
  printf("%ld %ld %ld %ld\n", wrong, fallback, kept_bad, lost);
  return 0;
}

// Host check of the integer-pipe binary64 routines (paper_2402_04514_gb300/csrc/softfp64.cuh) against the
// host's own IEEE 754 multiplication and addition: n seeded cases from several families, compared bit for
// bit (any NaN matches any NaN).  Prints the number of mismatches and exits non-zero if there is one.
#include "../paper_2402_04514_gb300/csrc/softfp64.cuh"
#include <cmath>
#include <cstdio>
#include <cstdlib>

static uint64_t st[2];
static uint64_t next() {  // xorshift128+
  uint64_t s1 = st[0];
  const uint64_t s0 = st[1];
  st[0] = s0;
  s1 ^= s1 << 23;
  st[1] = s1 ^ s0 ^ (s1 >> 17) ^ (s0 >> 26);
  return st[1] + s0;
}
static double make(uint64_t sign, int field, uint64_t frac) {
  return sf::dbl((sign << 63) | ((uint64_t)field << 52) | (frac & 0x000fffffffffffffull));
}
static bool same(double x, double y) { return std::isnan(x) ? std::isnan(y) : sf::bits(x) == sf::bits(y); }

int main(int argc, char** argv) {
  const long n = argc > 1 ? atol(argv[1]) : 1000000;
  st[0] = 0x9E3779B97F4A7C15ull ^ (argc > 2 ? strtoull(argv[2], 0, 10) : 0);
  st[1] = 0xBF58476D1CE4E5B9ull;
  static const double special[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 4.9e-324, -2.5e-320,
                                   2.2250738585072014e-308, 1.7976931348623157e308, 0.5};
  long bad_mul = 0, bad_add = 0, bad_pow2 = 0;
  for (long i = 0; i < n; ++i) {
    const uint64_t r1 = next(), r2 = next(), r3 = next();
    double a, b;
    switch (i % 8) {
      case 0:  // any bit patterns
        a = sf::dbl(r1), b = sf::dbl(r2);
        break;
      case 1:  // magnitudes near 1
        a = make(r3 & 1, 1000 + (int)((r3 >> 1) % 47), r1);
        b = make((r3 >> 8) & 1, 1000 + (int)((r3 >> 9) % 47), r2);
        break;
      case 2: {  // opposite signs, exponents within 4: cancellation
        a = make(r3 & 1, 1 + (int)((r3 >> 1) % 2046), r1);
        int f = (int)((sf::bits(a) >> 52) & 0x7ff) + (int)((r3 >> 20) % 9) - 4;
        f = f < 1 ? 1 : (f > 2046 ? 2046 : f);
        b = make(!(r3 & 1), f, ((r3 >> 40) & 1) ? (sf::bits(a) ^ (r2 & 0xff)) : r2);
        break;
      }
      case 3:  // an addend just below half an ulp, at it, or just above (ties)
        a = make(r3 & 1, 1023, r1 | 0xffffffffull);
        b = make((r3 >> 1) & 1, 1023 - 53 - (int)((r3 >> 2) % 3), (r2 >> 60) << 48);
        break;
      case 4:  // significands with trailing zeros
        a = make(r3 & 1, 1 + (int)((r3 >> 1) % 2046), r1 & ~((1ull << ((r3 >> 50) & 31)) - 1));
        b = make((r3 >> 12) & 1, 1 + (int)((r3 >> 13) % 2046), r2 & ~((1ull << ((r3 >> 40) & 31)) - 1));
        break;
      case 5:  // exponents near the subnormal range, 1 and the overflow threshold
        a = make(r3 & 1, (int)((r3 >> 1) % 3) * 1023 + (int)((r3 >> 3) % 40) - 20, r1);
        b = make((r3 >> 12) & 1, (int)((r3 >> 13) % 3) * 1023 + (int)((r3 >> 15) % 40) - 20, r2);
        break;
      case 6:  // zeros, infinities, NaN, subnormals and range ends against any operand
        a = (r3 & 1) ? special[r1 % 12] : make((r3 >> 1) & 1, 1 + (int)((r3 >> 2) % 2046), r1);
        b = special[r2 % 12];
        if (r3 & 2) {
          const double t = a;
          a = b, b = t;
        }
        break;
      default:
        if ((r3 >> 30) & 1) {  // products of short integers: exact products and ties
          a = ldexp((double)((r1 >> 37) | 1), (int)(r3 % 200) - 100);
          b = ldexp((double)((r2 >> 36) | 1), (int)((r3 >> 8) % 200) - 100);
          if (r3 & 1) b = -b;
        } else {  // b close to -a
          a = make(r3 & 1, 1023 + (int)((r3 >> 1) % 64) - 32, r1);
          b = -a * (1.0 + make(0, 1022 - (int)((r3 >> 10) % 60), r2));
        }
    }
    const double pm = sf::mul(a, b), hm = a * b, pa = sf::add(a, b), ha = a + b;
    if (!same(pm, hm) && bad_mul++ < 8) printf("mul %a * %a: host %a, integer %a\n", a, b, hm, pm);
    if (!same(pa, ha) && bad_add++ < 8) printf("add %a + %a: host %a, integer %a\n", a, b, ha, pa);
    int k = (int)(r3 % 121) - 60 + ((r3 >> 20) % 16 == 0 ? (int)((r3 >> 24) % 2045) - 1022 : 0);
    k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);  // the documented range of the scale
    const double ps = sf::mul_pow2(a, k), hs = a * ldexp(1.0, k);
    if (!same(ps, hs) && bad_pow2++ < 8) printf("pow2 %a * 2^%d: host %a, integer %a\n", a, k, hs, ps);
  }
  printf("cases %ld mul mismatches %ld add mismatches %ld pow2 mismatches %ld\n", n, bad_mul, bad_add, bad_pow2);
  return (bad_mul || bad_add || bad_pow2) ? 1 : 0;
}

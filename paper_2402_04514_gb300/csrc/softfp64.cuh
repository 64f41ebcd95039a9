// IEEE 754 binary64 multiplication and addition, rounded to nearest with ties to even, on the integer
// pipe.
//
// The GB300's FP64 pipe retires 2 thread-operations per clock per SM, 1/64 of the FP32 rate, while its
// integer pipes retire 64.  The sweep kernels are bound by the FP64 pipe with most of their issue slots
// free, so moving part of their FP64 products to these integer routines runs both pipes at once (the sum
// is here too; it costs about twice a product and the kernels keep their sums on the FP64 pipe).
// Every result is the correctly rounded IEEE result (the same bits as the hardware instruction), so a
// kernel gives the same results whichever of its operations take this path.  The routines follow the
// definition of the operations in IEEE 754 (form the exact result, then round it to nearest, ties to
// even) on the significands as integers.
//
// The integer path covers normal operands whose result is normal, and zeros.  Everything else (subnormal,
// infinite or NaN operands, a result at the ends of the exponent range) takes the hardware instruction, so
// that the special cases keep IEEE semantics exactly.  The header compiles as host C++ too, where the
// same integer code is checked against the host's own binary64 arithmetic.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SF_FN __host__ __device__ __forceinline__
#else
#define SF_FN static inline
#endif

namespace sf {

SF_FN uint64_t bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

SF_FN double dbl(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}

SF_FN uint32_t hiw(double x) { return (uint32_t)(bits(x) >> 32); }
SF_FN uint32_t low(double x) { return (uint32_t)bits(x); }
SF_FN double dbl2(uint32_t h, uint32_t l) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)h, (int)l);
#else
  return dbl(((uint64_t)h << 32) | l);
#endif
}

// The hardware operation for the special cases, in a function of its own that the common path calls only
// when it needs it.  A plain `a * b` under a rarely taken branch is executed speculatively or predicated
// by the compiler, which costs its FP64 issue slot on every call.  const: the calls read and write no
// memory, so that they stop no load reuse or reordering around them.
#if defined(__CUDA_ARCH__)
static __device__ __noinline__ __attribute__((const)) double hw_mul(double a, double b) { return a * b; }
static __device__ __noinline__ __attribute__((const)) double hw_add(double a, double b) { return a + b; }
#else
static inline double hw_mul(double a, double b) { return a * b; }
static inline double hw_add(double a, double b) { return a + b; }
#endif

// Everything below works on the 32-bit words of the operands, with the carries of the 64-bit additions
// and of the 106-bit product written out (PTX add.cc / addc, mad.cc / madc).
// fsr / fsl: the low / high word of the 64-bit (hi:lo) shifted right / left by s (0 <= s < 32).
SF_FN uint32_t fsr(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> (s & 31));
#endif
}
SF_FN uint32_t fsl(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, s);
#else
  return (uint32_t)(((((uint64_t)hi << 32) | lo) << (s & 31)) >> 32);
#endif
}
// x << (32 - s) for 0 <= s < 32, 0 for s = 0: the bits a right shift by s drops, at the top of the word
SF_FN uint32_t dropped(uint32_t x, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_lc(0u, x, 32u - s);
#else
  return s == 0 ? 0u : x << (32u - s);
#endif
}
SF_FN uint32_t clz32(uint32_t x) {  // 32 for x = 0
#if defined(__CUDA_ARCH__)
  return (uint32_t)__clz((int)x);
#else
  return x ? (uint32_t)__builtin_clz(x) : 32u;
#endif
}

// (h:l) = (xh:xl) + (yh:yl) and - (yh:yl) modulo 2^64
SF_FN void add64(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl, uint32_t& h, uint32_t& l) {
#if defined(__CUDA_ARCH__)
  asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;" : "=r"(l), "=r"(h) : "r"(xl), "r"(yl), "r"(xh), "r"(yh));
#else
  const uint64_t r = ((((uint64_t)xh) << 32) | xl) + ((((uint64_t)yh) << 32) | yl);
  h = (uint32_t)(r >> 32), l = (uint32_t)r;
#endif
}
SF_FN void sub64(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl, uint32_t& h, uint32_t& l) {
#if defined(__CUDA_ARCH__)
  asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, %4, %5;" : "=r"(l), "=r"(h) : "r"(xl), "r"(yl), "r"(xh), "r"(yh));
#else
  const uint64_t r = ((((uint64_t)xh) << 32) | xl) - ((((uint64_t)yh) << 32) | yl);
  h = (uint32_t)(r >> 32), l = (uint32_t)r;
#endif
}
// (h:l) += y with the carry out of bit 63 in c
SF_FN void inc64(uint32_t& h, uint32_t& l, uint32_t y, uint32_t& c) {
#if defined(__CUDA_ARCH__)
  asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, 0;\n\taddc.u32 %2, 0, 0;" : "+r"(l), "+r"(h), "=r"(c) : "r"(y));
#else
  const uint64_t x = (((uint64_t)h) << 32) | l, r = x + y;
  c = r < x, h = (uint32_t)(r >> 32), l = (uint32_t)r;
#endif
}
// the 106-bit product (ah:al)(bh:bl) of two 53-bit significands as four words w3..w0
SF_FN void mul53(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t& w3, uint32_t& w2, uint32_t& w1,
                 uint32_t& w0) {
#if defined(__CUDA_ARCH__)
  asm("mul.lo.u32 %0, %4, %6;\n\t"
      "mul.hi.u32 %1, %4, %6;\n\t"
      "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
      "madc.hi.u32 %2, %5, %6, 0;\n\t"
      "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
      "madc.hi.u32 %2, %4, %7, %2;\n\t"
      "mad.lo.cc.u32 %2, %5, %7, %2;\n\t"
      "madc.hi.u32 %3, %5, %7, 0;"
      : "=&r"(w0), "=&r"(w1), "=&r"(w2), "=&r"(w3)
      : "r"(al), "r"(ah), "r"(bl), "r"(bh));
#else
  const uint64_t p0 = (uint64_t)al * bl;
  uint64_t t = (uint64_t)ah * bl + (p0 >> 32);
  const uint64_t t2 = (uint64_t)al * bh + (uint32_t)t;
  const uint64_t u = (uint64_t)ah * bh + (t >> 32) + (t2 >> 32);
  w0 = (uint32_t)p0, w1 = (uint32_t)t2, w2 = (uint32_t)u, w3 = (uint32_t)(u >> 32);
#endif
}

// a * b.  With A, B the 53-bit significands (implicit bit included) the exact product P = A B lies in
// [2^104, 2^106); H = P >> 43 keeps its top 62 or 63 bits with the rest folded into bit 0 (sticky), a
// one-bit shift puts the leading bit at 62, and adding 0x1ff plus the bit at 10 rounds at bit 10 to
// nearest even (a carry out of the significand moves into the exponent field through the addition that
// assembles the result).
SF_FN double mul(double a, double b) {
  const uint32_t ha = hiw(a), la = low(a), hb = hiw(b), lb = low(b);
  const int ea = (int)((ha >> 20) & 0x7ffu), eb = (int)((hb >> 20) & 0x7ffu);
  const int e = ea + eb - 1023;  // exponent field of the product when A B < 2^105
  uint32_t w3, w2, w1, w0;
  mul53((ha & 0xfffffu) | 0x100000u, la, (hb & 0xfffffu) | 0x100000u, lb, w3, w2, w1, w0);
  uint32_t hh = fsr(w2, w3, 11), hl = fsr(w1, w2, 11) | (uint32_t)(((w1 & 0x7ffu) | w0) != 0u);
  const uint32_t top = hh >> 30;  // 1 when P >= 2^105
  hh = fsl(hl, hh, top ^ 1u);
  hl <<= (top ^ 1u);
  uint32_t c;
  inc64(hh, hl, 0x1ffu + ((hl >> 10) & 1u), c);
  const uint32_t sg = (ha ^ hb) & 0x80000000u;
  uint32_t rh = ((hh >> 10) + ((uint32_t)(e + (int)top - 1) << 20)) | sg, rl = fsr(hl, hh, 10);
  const bool zero = ((((ha << 1) | la) == 0u) | (((hb << 1) | lb) == 0u)) & (ea != 0x7ff) & (eb != 0x7ff);
  if (zero) rh = sg, rl = 0u;  // 0 x finite
  const bool ok = ((unsigned)(ea - 1) < 2046u) & ((unsigned)(eb - 1) < 2046u) & ((unsigned)(e - 1) < 2044u);
  if (__builtin_expect(!(ok | zero), 0)) return hw_mul(a, b);  // subnormal, infinite or NaN operand or result
  return dbl2(rh, rl);
}

// x * 2^k for -1022 <= k <= 1023 by adding k to the exponent field: exact for a normal x whose scaled
// value is normal, and for zeros; every other case takes the FP64 instruction.
SF_FN double mul_pow2(double x, int k) {
  const uint32_t h = hiw(x), l = low(x);
  const int ex = (int)((h >> 20) & 0x7ffu);
  const bool zero = ((h << 1) | l) == 0u;
  const bool ok = ((unsigned)(ex - 1) < 2046u) & ((unsigned)(ex + k - 1) < 2046u);
  if (__builtin_expect(!(ok | zero), 0)) return hw_mul(x, dbl2((uint32_t)(1023 + k) << 20, 0u));
  return zero ? x : dbl2(h + ((uint32_t)k << 20), l);
}

// a + b.  x is the operand of larger magnitude, X and Y the significands with the leading bit at 62; Y is
// shifted right by the exponent difference with the bits shifted out folded into bit 0 (sticky), which
// rounds like the exact value because bit 0 lies below the rounding position.  The sum or difference R
// is normalised to bit 63 by its leading-zero count and rounded at bit 11 to nearest even; a carry out of
// bit 63 there means the significand rounded up to 2^53.
SF_FN double add(double a, double b) {
  const uint32_t ha = hiw(a), la = low(a), hb = hiw(b), lb = low(b);
  const uint32_t mha = ha & 0x7fffffffu, mhb = hb & 0x7fffffffu;
  const bool sw = (mha < mhb) | ((mha == mhb) & (la < lb));
  const uint32_t xh = sw ? hb : ha, xl = sw ? lb : la, yh = sw ? ha : hb, yl = sw ? la : lb;
  const int ex = (int)((xh >> 20) & 0x7ffu), ey = (int)((yh >> 20) & 0x7ffu);
  const int d = ex - ey;
  const uint32_t s = d < 63 ? (uint32_t)d : 63u;
  const uint32_t Xh = fsl(xl, (xh & 0xfffffu) | 0x100000u, 10), Xl = xl << 10;
  const uint32_t Yh = fsl(yl, (yh & 0xfffffu) | 0x100000u, 10), Yl = yl << 10;
  // Y >> s with sticky: a word shift when s >= 32, then a funnel shift by s mod 32
  const bool ge = s >= 32u;
  const uint32_t L = ge ? Yh : Yl, Hw = ge ? 0u : Yh, sh = s & 31u;
  const uint32_t lostw = dropped(L, sh) | (ge ? Yl : 0u);
  const uint32_t Al = fsr(L, Hw, sh) | (uint32_t)(lostw != 0u), Ah = Hw >> sh;
  uint32_t Sh, Sl, Dh, Dl;
  add64(Xh, Xl, Ah, Al, Sh, Sl);
  sub64(Xh, Xl, Ah, Al, Dh, Dl);
  const bool sub = ((ha ^ hb) & 0x80000000u) != 0u;
  const uint32_t Rh = sub ? Dh : Sh, Rl = sub ? Dl : Sl;
  const bool hz = Rh == 0u;
  const uint32_t lz = hz ? 32u + clz32(Rl) : clz32(Rh);
  const uint32_t Th = hz ? Rl : Rh, Tl = hz ? 0u : Rl, t = lz & 31u;
  uint32_t Hh = fsl(Tl, Th, t), Hl = Tl << t, c;
  inc64(Hh, Hl, 0x3ffu + ((Hl >> 11) & 1u), c);
  uint32_t rh = (((Hh >> 11) | (c << 21)) + ((uint32_t)(ex - (int)lz) << 20)) | (xh & 0x80000000u);
  uint32_t rl = fsr(Hl, Hh, 11);
  const bool rz = hz & (Rl == 0u);
  const bool yz = (((yh << 1) | yl) == 0u);
  if (rz) rh = 0u, rl = 0u;  // exact cancellation: +0
  if (yz) {                  // a zero operand: x + 0 = x; -0 + -0 = -0
    const bool xz = (((xh << 1) | xl) == 0u);
    rh = xz ? (ha & hb) : xh, rl = xz ? 0u : xl;
  }
  const bool ok = (yz & (ex != 0x7ff)) | (((unsigned)(ey - 1) < 2046u) & (ex <= 2044) & (rz | (ex >= (int)lz)));
  if (__builtin_expect(!ok, 0)) return hw_add(a, b);  // subnormal, infinite or NaN operand or result
  return dbl2(rh, rl);
}

SF_FN double sub(double a, double b) { return add(a, dbl2(hiw(b) ^ 0x80000000u, low(b))); }

}  // namespace sf

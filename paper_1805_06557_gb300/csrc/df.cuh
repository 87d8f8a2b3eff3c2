// Double-float arithmetic on the FP32 pipe: a value is carried as hi + lo (two FP32 words,
// |lo| <= ulp(hi) / 2), products are split exactly by FMA (TwoProduct) and sums by Knuth's
// TwoSum, so that about 48 significand bits survive where FP64 arithmetic is a scarce pipe
// (GB300 issues about two FP64 FMAs per clock and SM, 128 FP32 ones).  Shared by the mixed REXI
// solve kernels and the double-float Legendre contractions.
#pragma once
#include <cuda_runtime.h>

namespace rexi {

// ---- double-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2) --------------------
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return df{s, e};
}
__device__ __forceinline__ df df_fast(float s, float e) {  // |s| >= |e|
  float h = s + e;
  return df{h, e - (h - s)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = df_two_sum(x.hi, y.hi);
  return df_fast(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_mul(df x, df y) {
  float p = __fmul_rn(x.hi, y.hi);  // never contracted into a following add
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
  return df_fast(p, e);
}
__device__ __forceinline__ df df_mulf(df x, float f) {
  float p = __fmul_rn(x.hi, f);
  float e = fmaf(x.hi, f, -p);
  e = fmaf(x.lo, f, e);
  return df_fast(p, e);
}
// Compensated dot product (Ogita, Rump & Oishi's Dot2): the running sum s is kept in FP32 and
// every rounding error -- of each product (TwoProduct by FMA) and of each addition (Knuth's
// TwoSum) -- together with the low words of double-float operands is gathered in one FP32 word
// err, so that s + err is as accurate as a sum formed in twice the working precision.
struct dot2 {
  float s, err;
};
// acc += (a_hi + a_lo) * b, b in FP32
__device__ __forceinline__ void dot2_add(dot2& acc, df a, float b) {
  const float p = __fmul_rn(a.hi, b);  // the rounded product itself enters the TwoSum
  const float ep = fmaf(a.hi, b, -p);
  const df t = df_two_sum(acc.s, p);
  acc.s = t.hi;
  acc.err = fmaf(a.lo, b, acc.err + (ep + t.lo));
}
// acc += (a_hi + a_lo) * (b_hi + b_lo)
__device__ __forceinline__ void dot2_add2(dot2& acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float ep = fmaf(a.hi, b.hi, -p);
  const df t = df_two_sum(acc.s, p);
  acc.s = t.hi;
  acc.err = fmaf(a.lo, b.hi, fmaf(a.hi, b.lo, acc.err + (ep + t.lo)));
}


// The same for a complex sum of (real double-float) x (complex double-float) terms, both
// components at once on Blackwell's packed FP32x2 instructions (FMUL2 / FFMA2 / FADD2 round
// each component as the scalar instruction does): the operation sequence of dot2_add2 per
// component, in half the instructions.  The complex factor comes as its high words (re, im)
// and its low words (re, im).
struct dot2c {
  float2 s, err;
};
__device__ __forceinline__ float2 f2n(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void dot2c_add(dot2c& acc, df a, float2 bhi, float2 blo) {
  const float2 ah = make_float2(a.hi, a.hi);
  const float2 p = __fmul2_rn(ah, bhi);
  const float2 ep = __ffma2_rn(ah, bhi, f2n(p));
  const float2 s = __fadd2_rn(acc.s, p);                      // TwoSum(acc.s, p)
  const float2 bb = __fadd2_rn(s, f2n(acc.s));
  const float2 e = __fadd2_rn(__fadd2_rn(acc.s, f2n(__fadd2_rn(s, f2n(bb)))), __fadd2_rn(p, f2n(bb)));
  acc.s = s;
  acc.err = __ffma2_rn(make_float2(a.lo, a.lo), bhi, __ffma2_rn(ah, blo, __fadd2_rn(acc.err, __fadd2_rn(ep, e))));
}
__device__ __forceinline__ dot2 dot2c_re(const dot2c& a) { return dot2{a.s.x, a.err.x}; }
__device__ __forceinline__ dot2 dot2c_im(const dot2c& a) { return dot2{a.s.y, a.err.y}; }

// ---- a double-float real with arithmetic operators (for code templated on its real type,
// such as the longitude FFT): sums by TwoSum, products by TwoProduct, both renormalised -------
struct dfr {
  float hi, lo;
  dfr() = default;
  __device__ __forceinline__ dfr(float h, float l) : hi(h), lo(l) {}
  // from FP64 (an FP64 conversion; constant arguments fold at compile time)
  __device__ __forceinline__ explicit dfr(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.hi, -a.lo); }
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  const df s = df_two_sum(a.hi, b.hi);
  const df r = df_fast(s.hi, s.lo + (a.lo + b.lo));
  return dfr(r.hi, r.lo);
}
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const df r = df_mul(df{a.hi, a.lo}, df{b.hi, b.lo});
  return dfr(r.hi, r.lo);
}
// by a sign (+1 or -1)
__device__ __forceinline__ dfr operator*(int s, dfr a) { return s > 0 ? a : -a; }

// ---- FP64 <-> double-float by the bit patterns (integer pipe; GB300's FP64 pipe, which the
// conversion instructions use, issues about 2 operations per clock and SM) -------------------
// the float with sign sgn, biased exponent be (1..254) and the 23 fraction bits below the
// leading one of r (r != 0), truncated
__device__ __forceinline__ float df_bits_float(unsigned sgn, int be, unsigned r) {
  const int lz = __clz(r);  // <= 31; the shift below moves the leading one to bit 32
  const unsigned frac = (unsigned)((((unsigned long long)r) << (lz + 1)) >> 9) & 0x7fffffu;
  return __uint_as_float(sgn | ((unsigned)be << 23) | frac);
}
// x = hi + lo: hi its leading 24 significand bits, lo the next 24 (both truncated; about 48 bits
// of x); values whose low word could leave the FP32 normal range (|x| < 2^-73, zeros and
// subnormals included) or whose high word would overflow take the FP64 route
__device__ __forceinline__ dfr dfr_from_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const int ef = e - 1023 + 127;  // FP32 biased exponent of the leading bit
  if (ef < 54 || ef > 254) return dfr(x);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;  // 52 stored fraction bits
  const float hi = __uint_as_float(sgn | ((unsigned)ef << 23) | (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & 0x1FFFFFFFu);  // the remaining 29 bits, weight 2^(e - 1075)
  if (r == 0) return dfr(hi, 0.f);
  // leading bit of r at position 31 - clz(r) >= 0: biased exponent ef - 52 + (31 - clz(r)) >= 2
  return dfr(hi, df_bits_float(sgn, ef - 52 + 31 - __clz(r), r));
}
// a float widened exactly to FP64 from its bits
__device__ __forceinline__ double df_widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ef = (b >> 23) & 0xff;
  if (ef == 0 || ef == 255) return (double)f;  // zero, subnormal, inf, nan
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(ef + 896) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

}  // namespace rexi

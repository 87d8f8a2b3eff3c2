// Conversions between binary64 and binary32 by their IEEE 754 bit layouts, on the integer pipe.
// On this GPU the F2F conversion instructions run on the FP64 pipe, at about two per clock and
// SM, and kernels that only move FP64 data in and out of FP32 arithmetic (the FP32 longitude
// FFT) are bound by it.  The integer paths cover every input whose result is a normal binary32 /
// binary64 number, and signed zeros; subnormal results, infinities and NaNs take the hardware
// conversion.
// Results equal the hardware's bit for bit: FP64 -> FP32 rounds to nearest, ties to even; FP32
// -> FP64 is exact.  Plain C++ apart from the qualifiers, so the host test compiles it too.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define CVT_HD __host__ __device__ __forceinline__
#else
#define CVT_HD inline
#endif

namespace cvt {

CVT_HD uint64_t bits64(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  memcpy(&u, &d, sizeof u);
  return u;
#endif
}
CVT_HD double from_bits64(uint32_t hi, uint32_t lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &u, sizeof d);
  return d;
#endif
}
CVT_HD uint32_t bits32(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  return u;
#endif
}
CVT_HD float from_bits32(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
#endif
}

// binary64 -> binary32, round to nearest, ties to even.  binary64 = sign | e11 | 52 mantissa
// bits (bias 1023), binary32 = sign | e8 | 23 bits (bias 127): e8 = e11 - 896.  The fast path
// takes e11 in [897, 1150], i.e. e8 in [1, 254] before rounding.
CVT_HD float f64_to_f32(double d) {
  const uint64_t b = bits64(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e11 = (hi >> 20) & 0x7ffu;
  if (e11 - 897u > 253u) {
    if (((hi << 1) | lo) == 0u) return from_bits32(hi);  // +-0 (hi holds only the sign)
    return (float)d;
  }
  // bits 60..29 of d: the low nine exponent bits above the 23 leading mantissa bits
  uint32_t t = (hi << 3) | (lo >> 29);
  // exponent field minus 896, modulo 2^9 (896 = 384 mod 512); the result e8 <= 254 leaves bit
  // 31 clear for the sign
  t = (t - 0xC0000000u) | (hi & 0x80000000u);
  // the 29 dropped bits: round up above half, at half when the kept last bit is odd; a carry
  // out of the mantissa raises the exponent (254 -> 255 gives infinity, as rounding overflows)
  const uint32_t rest = lo & 0x1fffffffu;
  t += (rest + 0x0fffffffu + (t & 1u)) >> 29;
  return from_bits32(t);
}

// binary32 -> binary64, exact.  The fast path takes e8 in [1, 254] (normal numbers).
CVT_HD double f32_to_f64(float f) {
  const uint32_t u = bits32(f);
  const uint32_t e8 = (u >> 23) & 0xffu;
  if (e8 - 1u > 253u) {
    if ((u << 1) == 0u) return from_bits64(u, 0u);  // +-0
    return (double)f;
  }
  // exponent + 896 and the 20 leading mantissa bits in the high word, the last 3 in the low one
  const uint32_t hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
  return from_bits64(hi, u << 29);
}

}  // namespace cvt

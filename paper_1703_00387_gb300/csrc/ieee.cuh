// Float conversions by integer operations on the IEEE-754 bit layouts.
//
// GB300's float64 pipe issues two lanes per clock per SM, and widening a
// float to double runs there: converting every element of a 128 x 256 tile
// in a GEMM epilogue measured ~8 us per launch. (Narrowing by integer fields
// measured slower than the hardware conversion inside the fused W-step, so
// that kernel keeps the hardware one.) These helpers build the result from the
// sign, exponent and fraction fields with integer operations (the integer
// pipe is 32 times wider) for normal numbers, and leave zeros, subnormals,
// infinities, NaNs and out-of-range exponents to the hardware conversion
// (both return signed zeros themselves: they are common as padding).
// Both are exact restatements of the format's definition: widening copies
// the fraction; narrowing rounds the fraction to nearest, ties to even.
#pragma once
#include <stdint.h>

#include <cuda_bf16.h>

namespace osmps {

// (double)x, exactly.
__device__ __forceinline__ double f32_to_f64(float x) {
  const uint32_t u = __float_as_uint(x);
  if ((u << 1) == 0) return __longlong_as_double((long long)((uint64_t)(u >> 31) << 63));  // +-0
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)x;  // zero, subnormal, inf, nan
  const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                        ((uint64_t)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// (float)x, rounded to nearest with ties to even.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  if ((b << 1) == 0) return __uint_as_float((uint32_t)(b >> 63) << 31);  // +-0
  const int E = (int)((b >> 52) & 0x7FFu);
  const int ef = E - 896;  // float biased exponent
  if (ef < 1 || ef > 253) return (float)x;  // float subnormals, overflow, zero, inf, nan
  const uint64_t frac = b & 0xFFFFFFFFFFFFFull;
  const uint32_t keep = (uint32_t)(frac >> 29);            // 23 fraction bits kept
  const uint32_t rest = (uint32_t)(frac & 0x1FFFFFFFu);    // 29 bits dropped
  const uint32_t half = 0x10000000u;
  uint32_t mag = ((uint32_t)ef << 23) | keep;
  mag += (rest > half || (rest == half && (keep & 1u))) ? 1u : 0u;  // a carry moves into the exponent
  return __uint_as_float((uint32_t)(b >> 63) << 31 | mag);
}

// (float)x rounded to odd: the fraction truncated to 23 bits, its last bit
// set when any dropped bit was set. Rounding that to nearest-even at 7
// fraction bits (bf16) equals rounding x to bf16 directly, since float keeps
// more than 7 + 2 bits (the round-to-odd argument of Boldo and Melquiond,
// "Emulation of FMA and correctly rounded sums: proved algorithms using
// rounding to odd", IEEE Trans. Computers 57 (2008)). Normal floats only:
// returns false (and leaves *out) when x is zero, subnormal, infinite, NaN
// or outside the float exponent range.
__device__ __forceinline__ bool f64_to_f32_odd(double x, float* out) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7FFu) - 896;
  if (ef < 1 || ef > 254) return false;
  const uint64_t frac = b & 0xFFFFFFFFFFFFFull;
  const uint32_t keep = (uint32_t)(frac >> 29) | ((frac & 0x1FFFFFFFu) != 0 ? 1u : 0u);
  *out = __uint_as_float((uint32_t)(b >> 63) << 31 | ((uint32_t)ef << 23) | keep);
  return true;
}

// x rounded to nearest-even bf16: through float32 rounded to odd (integer
// fields, exact under the double rounding), then the float-to-bf16
// conversion; signed zeros directly, the hardware conversion where x is not
// a normal float.
__device__ __forceinline__ __nv_bfloat16 f64_to_bf16_rn(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  if ((b << 1) == 0) return __ushort_as_bfloat16((unsigned short)((b >> 48) & 0x8000u));
  float xo;
  return f64_to_f32_odd(x, &xo) ? __float2bfloat16_rn(xo) : __double2bfloat16(x);
}

}  // namespace osmps

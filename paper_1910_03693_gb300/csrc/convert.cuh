// FP64 -> FP32 rounding (IEEE-754 round to nearest, ties to even) from the
// bit fields, on the integer pipe.  On GB300 the hardware conversion issues
// on the FP64 pipe, which the FP64-bound Arnoldi kernels already saturate.
// binary64: sign, 11-bit exponent (bias 1023), 52-bit fraction; binary32:
// sign, 8-bit exponent (bias 127), 23-bit fraction.  A normal binary32 result
// needs the biased binary64 exponent in [897, 1150]; the 29 dropped fraction
// bits decide the rounding, and a carry out of the fraction moves into the
// exponent (rounding the largest finite values up gives infinity, as IEEE
// rounding does).  Zeros keep their sign; every other input outside that
// range (subnormal results, infinities, NaN) takes the hardware conversion.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

namespace frgb {

__device__ __forceinline__ float f32_from_f64_rn(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof(b));
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  if ((b << 1) == 0) {   // +0 or -0
    const uint32_t z = sign;
    float f;
    memcpy(&f, &z, sizeof(f));
    return f;
  }
  const int e = (int)((b >> 52) & 0x7ffu);
  if (e < 897 || e > 1150) return __double2float_rn(x);
  const uint64_t frac = b & 0xFFFFFFFFFFFFFull;
  uint32_t r = sign | ((uint32_t)(e - 896) << 23) | (uint32_t)(frac >> 29);
  const uint64_t rem = frac & 0x1FFFFFFFull, half = 0x10000000ull;
  if (rem > half || (rem == half && (r & 1u))) r += 1u;
  float f;
  memcpy(&f, &r, sizeof(f));
  return f;
}

}  // namespace frgb

// FP64 <-> FP32 conversions of the mixed-precision Jacobian, written with
// integer operations on the bit patterns.  On this part the FP64 pipe, the
// binding resource of the Jacobian kernels, also executes the hardware
// conversions; these keep them on the integer pipe.  Plain C++ as well, so
// that the generated mixed-precision code can be checked on the CPU with the
// same conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define QSS_CVT_FN __host__ __device__ __forceinline__
#else
#define QSS_CVT_FN static inline
#endif

// double -> float, rounded to nearest (ties away from zero).  |x| below the
// smallest normal float (2^-126) gives a signed zero; |x| beyond the largest
// float, and infinities, give infinity; NaN stays NaN.
QSS_CVT_FN float qss_f32(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int eb = (int)((hi >> 20) & 0x7ffu);
  const int e = eb - 1023 + 127;                          // the float's biased exponent
  const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the top 23 mantissa bits
  // the rounding increment carries into the exponent field when the
  // mantissa is all ones (and to infinity from the largest binade)
  uint32_t r = (sign | ((uint32_t)e << 23) | mant) + ((lo >> 28) & 1u);
  if (e <= 0) r = sign;
  if (e >= 255) r = sign | 0x7f800000u | ((eb == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
  float f;
  memcpy(&f, &r, 4);
  return f;
}

// float -> double, exact for normal floats; zeros and subnormals give a
// signed zero, infinities and NaN stay so.
QSS_CVT_FN double qss_f64(float f) {
  uint32_t fb;
  memcpy(&fb, &f, 4);
  const uint32_t sign = fb & 0x80000000u, ef = (fb >> 23) & 0xffu, m = fb & 0x7fffffu;
  uint32_t hi = sign | ((ef + 896u) << 20) | (m >> 3);
  uint32_t lo = m << 29;
  if (ef == 0) hi = sign, lo = 0;
  if (ef == 255) hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double x;
  memcpy(&x, &b, 8);
  return x;
}

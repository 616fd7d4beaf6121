// Device math used by the generated mechanism code (sm_103a, FP64).
//
// The generated straight-line code calls only qss_exp, qss_log and qss_rcp for
// its non-elementary operations; everything else is add/mul/fma.  On this part
// the FP64 pipe is the binding resource (its rate is about 1/60 of FP32), so
// these functions are written to spend few FP64 instructions and to do their
// bookkeeping (rounding to an integer, table index, exponent scaling, range
// checks) in the integer pipe.
#pragma once
#include <cuda_runtime.h>

#include "qss_exp_table.inc"

__device__ __forceinline__ double qss_rcp(double x) { return __drcp_rn(x); }

// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989), 128 entries:
//   x = (128 k + j) ln2/128 + r,  |r| <= ln2/256,
//   exp(x) = 2^k * 2^(j/128) * (1 + q),  q = r + r^2/2 + ... + r^5/120.
// n = 128 k + j is obtained by adding 1.5 * 2^52 (its low word is then n);
// ln2/128 is split so that n * hi is exact.  The truncation error of the
// polynomial is below 6e-19 relative; the result is within a few ulp of
// exp(x).  |x| >= 708 and NaN take the library exp (subnormal and overflowing
// results, never reached by the workloads' arguments).  10 FP64 instructions.
__device__ __forceinline__ double qss_exp_table(double x) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x40862000) return exp(x);
  const double shifter = 6755399441055744.0;   // 1.5 * 2^52
  const double t = fma(x, QSS_EXP_INV_STEP, shifter);
  const int n = __double2loint(t);
  const double nd = t - shifter;
  double r = fma(-nd, QSS_EXP_STEP_HI, x);
  r = fma(-nd, QSS_EXP_STEP_LO, r);
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  const double q = p * r;
  const double tj = __ldg(&qss_exp2_tab[n & 127]);
  const double res = fma(tj, q, tj);
  const int scale = (int)((unsigned)(n >> 7) << 20);   // k in the exponent field
  return __hiloint2double(__double2hiint(res) + scale, __double2loint(res));
}

#ifdef QSS_LIBRARY_EXP
__device__ __forceinline__ double qss_exp(double x) { return exp(x); }
#else
__device__ __forceinline__ double qss_exp(double x) { return qss_exp_table(x); }
#endif
__device__ __forceinline__ double qss_log(double x) { return log(x); }

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
#include "qss_log_table.inc"

__device__ __forceinline__ double qss_rcp(double x) { return __drcp_rn(x); }

// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989), 256 entries:
//   x = (256 k + j) ln2/256 + r,  |r| <= ln2/512,
//   exp(x) = 2^k * 2^(j/256) * (1 + q),  q = r + r^2/2 + r^3/6 + r^4/24.
// n = 256 k + j is obtained by adding 1.5 * 2^52 (its low word is then n);
// ln2/256 is split so that n * hi is exact.  The truncation error of the
// polynomial is below 4e-17 relative; the result is within about one ulp of
// exp(x).  |x| >= 708 and NaN take the library exp (subnormal and overflowing
// results, never reached by the workloads' arguments).  9 FP64 instructions.
__device__ __forceinline__ double qss_exp_table(double x) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x40862000) return exp(x);
  const double shifter = 6755399441055744.0;   // 1.5 * 2^52
  const double t = fma(x, QSS_EXP_INV_STEP, shifter);
  const int n = __double2loint(t);
  const double nd = t - shifter;
  double r = fma(-nd, QSS_EXP_STEP_HI, x);
  r = fma(-nd, QSS_EXP_STEP_LO, r);
  double p = fma(r, 1.0 / 24.0, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  const double q = p * r;
  const double tj = __ldg(&qss_exp2_tab[n & 255]);
  const double res = fma(tj, q, tj);
  const int scale = (int)((unsigned)(n >> 8) << 20);   // k in the exponent field
  return __hiloint2double(__double2hiint(res) + scale, __double2loint(res));
}

// log(x) for normal positive x by table lookup and an exact reduction (the
// table and its derivation are in gen_log_table.py):
//   x = 2^m y, y in [b, 2b), b ~ sqrt(1/2);  cell j of y from its bit pattern;
//   r = y c_j - 1 (exact: c_j has 9 significant bits), |r| <= 2^-8;
//   log x = (m ln2_hi + L_hi) + ((m ln2_lo + L_lo) + log1p(r)),
// the first sum exact, log1p(r) = r + r^2 q(r) with the Taylor terms up to
// r^7 (truncation below 2^-59 relative).  m, j and y come from integer
// operations on the bits.  Zero, negative, subnormal, infinite and NaN
// arguments take the library log.  13 FP64 instructions.
__device__ __forceinline__ double qss_log_table(double x) {
  const long long xb = __double_as_longlong(x);
  if ((unsigned long long)(xb - 0x0010000000000000LL) >= 0x7fe0000000000000ULL) return log(x);
  const long long off = xb - QSS_LOG_BASE_BITS;
  const long long m = off >> 52;                       // arithmetic shift
  const double y = __longlong_as_double(xb - (m << 52));
  const int j = (int)((off >> 44) & 255);
  const double c = __ldg(&qss_log_tab[j][0]);
  const double lhi = __ldg(&qss_log_tab[j][1]);
  const double llo = __ldg(&qss_log_tab[j][2]);
  const double r = fma(y, c, -1.0);
  const double r2 = r * r;
  // q(r) = -1/2 + r/3 - r^2/4 + r^3/5 - r^4/6 + r^5/7
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -0.25);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double p = fma(r2, q, r);
  const double md = (double)(int)m;
  const double head = fma(md, QSS_LOG_LN2_HI, lhi);
  const double tail = fma(md, QSS_LOG_LN2_LO, llo) + p;
  return head + tail;
}

#ifdef QSS_LIBRARY_EXP
__device__ __forceinline__ double qss_exp(double x) { return exp(x); }
#else
__device__ __forceinline__ double qss_exp(double x) { return qss_exp_table(x); }
#endif
#ifdef QSS_LIBRARY_LOG
__device__ __forceinline__ double qss_log(double x) { return log(x); }
#else
__device__ __forceinline__ double qss_log(double x) { return qss_log_table(x); }
#endif

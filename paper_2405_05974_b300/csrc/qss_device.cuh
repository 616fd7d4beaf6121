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

// QSS_DEBUG builds (-DQSS_DEBUG=1): the kernels check every index they form
// into the caller's arrays and into the Newton scratch against the extents
// they were given, before the access; a violation records a code in the
// module's status word (the first one wins) and the thread (a warp, where the
// condition is warp-uniform) returns without the access.  No trap: the
// context stays usable; qss_debug_status reads and clears the word.  Release
// builds compile the checks away.
#if defined(QSS_DEBUG) && QSS_DEBUG
__device__ int qss_debug_word;
#define QSS_DBG_CHECK(cond, code)                  \
  do {                                             \
    if (!(cond)) {                                 \
      atomicCAS(&qss_debug_word, 0, (int)(code));  \
      return;                                      \
    }                                              \
  } while (0)
#else
#define QSS_DBG_CHECK(cond, code) do { } while (0)
#endif

// 1/x from a single-precision seed refined by one cubic step of the
// reciprocal iteration (the order-3 form of Newton-Raphson for 1/x; J.-M.
// Muller et al., Handbook of Floating-Point Arithmetic, 2nd ed. 2018,
// Sec. 4.7):
//   y0 ~ 1/x to about 2^-20 (rcp.approx.f32 of the leading 20 mantissa bits,
//   the exponent and sign put back with integer operations),
//   e = 1 - x y0 (exact up to one rounding in the fma),
//   y = y0 (1 + e + e^2) = y0 + y0 (e + e^2),
// whose truncation error e^3 is below 2^-59, so y is within one ulp of 1/x
// (a CPU emulation with the seed perturbed by +-1 float ulp rounds 99.97 %
// of random arguments correctly).  Zero, subnormal, infinite and NaN
// arguments, and |x| >= 2^1021 (subnormal results), take the library
// reciprocal.  3 FP64 instructions.
__device__ __forceinline__ double qss_rcp(double x) {
  const unsigned hx = (unsigned)__double2hiint(x);
  const unsigned eb = (hx >> 20) & 0x7ffu;
  if (eb - 1u >= 0x7fcu) return __drcp_rn(x);
  const float f = __uint_as_float(0x3f800000u | ((hx & 0xfffffu) << 3));
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));
  // r in (1/2, 1]: its float exponent field minus 127, plus 1023 - (eb - 1023),
  // is the double's exponent field; the float mantissa fills the top 23 bits
  const unsigned rb = __float_as_uint(r);
  const unsigned yhi = (hx & 0x80000000u) | ((rb >> 3) + ((1919u - eb) << 20));
  const double y0 = __hiloint2double((int)yhi, (int)(rb << 29));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// An integer with |n| < 2^24 as a double, off the FP64 pipe (which also
// executes the int -> double conversion on this part): the float conversion
// is exact for such n, and the float's fields widen to the double's with
// integer operations -- sign kept, exponent re-biased by 1023 - 127 = 896
// (0x38000000 in the high word), the 23 mantissa bits split 20 / 3 between
// the high and low words.  Zero has no biased exponent and is selected.
__device__ __forceinline__ double qss_small_int_to_double(int n) {
  const unsigned fb = __float_as_uint((float)n);
  const unsigned hi = (fb & 0x80000000u) | (((fb & 0x7fffffffu) >> 3) + 0x38000000u);
  return __hiloint2double(fb ? (int)hi : 0, (int)(fb << 29));
}

// exp(x) by Tang's table-driven method (ACM TOMS 15(2), 1989), 2048 entries:
//   x = (2048 k + j) ln2/2048 + r,  |r| <= ln2/4096,
//   exp(x) = 2^k * 2^(j/2048) * (1 + q),  q = r + r^2/2 + r^3/6.
// n = 2048 k + j is obtained by adding 1.5 * 2^52 (its low word is then n);
// ln2/2048 is split so that n * hi is exact.  The truncation error of the
// cubic is below 3.5e-17 relative; the result is within one ulp of exp(x)
// (CPU emulation of these operations against exact values).  The 16 KB table
// stays in L1.  |x| >= 708 and NaN take the library exp (subnormal and
// overflowing results, never reached by the workloads' arguments).  n as a
// double comes from integer operations (qss_small_int_to_double), not from
// t - 1.5 * 2^52.  7 FP64 instructions.
__device__ __forceinline__ double qss_exp_table(double x) {
  const int hx = __double2hiint(x) & 0x7fffffff;
  if (hx >= 0x40862000) return exp(x);
  const double shifter = 6755399441055744.0;   // 1.5 * 2^52
  const double t = fma(x, QSS_EXP_INV_STEP, shifter);
  const int n = __double2loint(t);             // |n| < 708 * 2048 / ln2 < 2^21
  const double nd = qss_small_int_to_double(n);
  double r = fma(-nd, QSS_EXP_STEP_HI, x);
  r = fma(-nd, QSS_EXP_STEP_LO, r);
  double p = fma(r, 1.0 / 6.0, 0.5);
  p = fma(p, r, 1.0);
  const double q = p * r;
  const double tj = __ldg(&qss_exp2_tab[n & (QSS_EXP_L - 1)]);
  const double res = fma(tj, q, tj);
  const int scale = (int)((unsigned)(n >> 11) << 20);   // k in the exponent field
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
// arguments take the library log.  12 FP64 instructions (m as a double from
// integer operations).
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
  const double md = qss_small_int_to_double((int)m);   // -1022 <= m <= 1024
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

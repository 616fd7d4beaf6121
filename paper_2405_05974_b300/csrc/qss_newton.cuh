// Implicit (backward-Euler) step kernels around a generated mechanism body.
//
// Newton on G(phi) = phi - phi0 - dt f(phi), phi = (C, T), f = (wdot, Tdot) at
// constant volume, with the matrix M = I - dt J where J is the analytic
// Jacobian, re-evaluated every iteration.  phi0 is the initial state, or a
// constant term supplied by the caller (a BDF2 substep of qss_integrate:
// phi0 = a1 phi_n + a2 phi_n-1, dt = beta h); the iteration starts from the
// state either way.  One Newton iteration is two
// launches over the cells that are still iterating (a compacted list):
//   qss_jac_kernel (list mode)   f and J at the current iterate, one thread
//                                per cell (the generated body is compiled in
//                                this one kernel only)
//   qss_newton_update_*_kernel   M = I - dt J, factorisation, solve, update of
//                                phi, convergence test, next list
// The host enqueues max_iter iterations without synchronising: once a cell
// has converged or failed it leaves the list, so later launches cost only what
// the remaining cells need.
//
// The update kernel solves one cell's system at a time per warp (the warps
// stride over the active list, so a nearly empty list costs one cell per
// warp), with partial pivoting (warp arg-max, lowest index on ties) and the
// right-hand side eliminated with the matrix.
//   update_fp64    elimination and solve in FP64, in place in shared memory,
//                  the trailing block of each step split evenly over the
//                  lanes (qss_smem_solve_fp64).
//   update_fp32ir  M equilibrated by powers of two (rows, then columns),
//                  factorisation in FP32 as a compact loop (qss_solve_fp32ir);
//                  the solution refined with FP64 residuals g - M x (M from
//                  the FP64 copy in shared memory, staged once per cell)
//                  until the correction is below refine_tol relative, stops
//                  shrinking, or after max_refine sweeps; a zero or
//                  non-finite FP32 pivot (or a non-finite correction) sends
//                  that cell's solve to the FP64 elimination instead.
// Rates, equilibrium constants, the QSS solve, J, M and the Newton residual
// are FP64 in both forms.
//
// Scratch (global memory, one chunk of `cells` cells, leading dimension sld;
// s = cell - c0, t = position in the active list):
//   M64[(t/4) 4 QSS_JAC_NNZ + 4 e + t%4]  J of the t-th active cell (e = i NN + j,
//                                        or the CSR position), four cells
//                                        interleaved (whole-sector stores,
//                                        sectors shared by consecutive warps)
//   F [k * sld + t]                       f at the current iterate (written by
//                                        the Jacobian kernel in list mode)
//   PHI, PHI0 [k * sld + s]               iterate, constant term of G
//   ACT, ST, IT [s]                       active flag, status, iterations
//   LIST[2][sld], NACT[2]                 active lists (double-buffered)
#pragma once

#include <type_traits>

#define QSS_CELL_CONVERGED 0
#define QSS_CELL_MAXITER 1
#define QSS_CELL_NONFINITE 2
#define QSS_CELL_SINGULAR 3

#if QSS_NN > 64
#error "the warp-cooperative Newton solver supports at most 63 transported species"
#endif
#define QSS_NSLOT ((QSS_NN + 31) / 32)
// warps per update block: both forms stage one matrix per warp in shared
// memory (NN x (NN+1) doubles), within the 48 KB static limit
#define QSS_MSTRIDE (QSS_NN + 1)
#define QSS_MBYTES (QSS_NN * QSS_MSTRIDE * 8)
#define QSS_UPD_WARPS (QSS_MBYTES * 4 <= 44000 ? 4 : (QSS_MBYTES * 2 <= 44000 ? 2 : 1))
// the FP32_IR form also keeps its FP32 factors (NN x (NN+1) floats) per warp
#define QSS_M32BYTES (QSS_MBYTES + QSS_NN * QSS_MSTRIDE * 4 + QSS_NN * 24 + 8)
#define QSS_UPD_WARPS32 (QSS_M32BYTES * 4 <= 44000 ? 4 : (QSS_M32BYTES * 2 <= 44000 ? 2 : 1))

__device__ __forceinline__ bool qss_finite(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// |x| ordered as an integer (no FP64 instruction): valid for finite and inf.
__device__ __forceinline__ long long qss_absbits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// Exponent e with 2^e <= |x| < 2^(e+1) for normal x; -1100 for zero/subnormal.
__device__ __forceinline__ int qss_ilogb(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7ff;
  return ex == 0 ? -1100 : ex - 1023;
}

__device__ __forceinline__ double qss_pow2(int e) {   // 2^e, e clamped to [-1000, 1000]
  e = max(min(e, 1000), -1000);
  return __hiloint2double((e + 1023) << 20, 0);
}

// Magnitude key for pivot search (an integer, so that the comparisons and the
// warp reduction stay off the FP64 pipe).
__device__ __forceinline__ long long qss_key(double x) { return qss_absbits(x); }
__device__ __forceinline__ long long qss_key(float x) {
  return (long long)(__float_as_int(x) & 0x7fffffff);
}

__device__ __forceinline__ double qss_shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float qss_shfl(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_newton_setup_kernel(long long cells, long long c0, long long ld, const double* __restrict__ rho,
                        const double* __restrict__ T, const double* __restrict__ Y,
                        double* __restrict__ PHI, double* __restrict__ PHI0, int* __restrict__ ACT,
                        int* __restrict__ ST, int* __restrict__ IT, int* __restrict__ LIST,
                        int* __restrict__ NACT, long long sld, const int* __restrict__ ncap,
                        const double* __restrict__ P0, long long p0ld) {
  // ncap (optional): a device-side cell count that lowers `cells`, so that a
  // launch sequence captured for a size bucket serves any smaller batch.
  // P0 (optional): the constant term of G, P0[k * p0ld + c] (a multistep
  // formula's combination of past states); otherwise it is the state.
  if (ncap) cells = min(cells, (long long)*ncap);
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  QSS_DBG_CHECK(cells <= sld, 4);
  if (s == 0) { NACT[0] = (int)cells; NACT[1] = 0; }
  if (s >= cells) return;
  const long long c = c0 + s;
  QSS_DBG_CHECK(c < ld && (!P0 || c < p0ld), 5);
  const double r = rho[c];
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) {
    const double v = r * Y[k * ld + c] * qss_inv_W[k];
    PHI[k * sld + s] = v;
    PHI0[k * sld + s] = P0 ? P0[k * p0ld + c] : v;
  }
  PHI[QSS_N * sld + s] = T[c];
  PHI0[QSS_N * sld + s] = P0 ? P0[QSS_N * p0ld + c] : T[c];
  ACT[s] = 1;
  ST[s] = QSS_CELL_MAXITER;
  IT[s] = 0;
  LIST[s] = (int)s;
}

struct QssNewtonOpts {
  int max_iter;
  double rtol, atol_C, atol_T;
  int max_refine;
  double refine_tol;
};

// FP64 solve of one cell's Newton system M x = g by one warp, in place in the
// warp's shared-memory copy of the augmented matrix [M | g] (row r at
// Ms[r * QSS_MSTRIDE], g in column QSS_NN).  Gaussian elimination with
// partial pivoting (largest |a| in the column, lowest row on ties) and row
// exchanges; the pivot row is scaled by 1/pivot (unit upper triangle, so that
// back substitution needs no division), and the trailing block of each step,
// rows k+1.. x columns k+1..NN, is split evenly over the 32 lanes (entry e =
// lane + 32 m of the block, its row and column advanced incrementally), so
// every lane does ~1/32 of the n^3/3 FMAs whatever n is.  Multipliers are
// not kept (g is eliminated with the matrix); entries left of the diagonal
// become don't-care values and are never read.  The loops are rolled: the
// FP64 pipe, not instruction fetch, must be the bound (a fully unrolled
// register form of this solve was fetch-bound on B300, 74 stall cycles per
// issue waiting for instructions).  On return column QSS_NN holds x.  Returns
// false on an all-zero pivot column.
__device__ __forceinline__ bool qss_smem_solve_fp64(double* __restrict__ Ms, const int lane) {
  const unsigned FULL = 0xffffffffu;
#pragma unroll 1
  for (int k = 0; k < QSS_NN; ++k) {
    long long best = -1;
    int brow = QSS_NN;
    for (int i = k + lane; i < QSS_NN; i += 32) {
      const long long key = qss_key(Ms[i * QSS_MSTRIDE + k]);
      if (key > best) { best = key; brow = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(FULL, best, o);
      const int orow = __shfl_xor_sync(FULL, brow, o);
      if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
    }
    if (best <= 0) return false;
    double* __restrict__ rk = Ms + k * QSS_MSTRIDE;
    if (brow != k) {   // warp-uniform
      double* __restrict__ rp = Ms + brow * QSS_MSTRIDE;
      for (int c = k + lane; c <= QSS_NN; c += 32) {
        const double v = rk[c];
        rk[c] = rp[c];
        rp[c] = v;
      }
      __syncwarp();
    }
    const double inv = qss_rcp(rk[k]);
    for (int c = k + 1 + lane; c <= QSS_NN; c += 32) rk[c] *= inv;
    __syncwarp();
    // trailing block: W = NN - k columns (k+1 .. NN), NN - 1 - k rows
    const int W = QSS_NN - k, E = (QSS_NN - 1 - k) * W;
    const int di = 32 / W, dj = 32 - di * W;
    int i = k + 1 + lane / W, j = k + 1 + (lane - (lane / W) * W);
#pragma unroll 4
    for (int e = lane; e < E; e += 32) {
      double* __restrict__ ri = Ms + i * QSS_MSTRIDE;
      ri[j] = fma(-ri[k], rk[j], ri[j]);
      i += di;
      j += dj;
      if (j > QSS_NN) { j -= W; ++i; }
    }
    __syncwarp();
  }
  // back substitution, column oriented: x_k is final once the columns right
  // of k have been subtracted
#pragma unroll 1
  for (int k = QSS_NN - 1; k > 0; --k) {
    const double xk = Ms[k * QSS_MSTRIDE + QSS_NN];
    for (int i = lane; i < k; i += 32)
      Ms[i * QSS_MSTRIDE + QSS_NN] = fma(-Ms[i * QSS_MSTRIDE + k], xk, Ms[i * QSS_MSTRIDE + QSS_NN]);
    __syncwarp();
  }
  return true;
}

// Bit-level helpers of the FP32-IR solve: scalings by powers of two and the
// conversions between the two precisions are exponent-field arithmetic on the
// integer pipe (on this part every FP64-pipe instruction, even a conversion,
// occupies the pipe for a whole warp).

// float(x * 2^-s), mantissa truncated to 24 bits; 0 when x is zero or
// subnormal or the result is below FLT_MIN.  The caller keeps the result
// below 2^128.
__device__ __forceinline__ float qss_scaled_float(double x, int s) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 - s;
  const unsigned fb = (hi & 0x80000000u) | ((unsigned)(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  return (e < -126 || (hi & 0x7ff00000u) == 0) ? 0.0f : __uint_as_float(fb);
}

// (double)f * 2^k, exact; f normal or zero.  An exponent outside the normal
// double range (never reached by the equilibrated systems) takes the FP64
// multiply.
__device__ __forceinline__ double qss_float_to_double_scaled(float f, int k) {
  const unsigned b = __float_as_uint(f);
  const int ef = (int)((b >> 23) & 0xffu);
  const int ed = ef + 896 + k;
  if (ef == 0) return 0.0;
  if (ed < 1 || ed > 2046) return (double)f * qss_pow2(k);
  const unsigned hi = (b & 0x80000000u) | ((unsigned)ed << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(b << 29));
}

// 2^-s as a float (0 below FLT_MIN)
__device__ __forceinline__ float qss_pow2f_neg(int s) {
  return s > 126 ? 0.0f : __uint_as_float((unsigned)(127 - s) << 23);
}

// Rows of the last lane slot when it is at most half full (n = 33..48): the
// FP64 residual of those rows is spread over the whole warp, QSS_R2 lanes
// per column stride, instead of running on the few lanes that own them.
#define QSS_RLAST (QSS_NN - 32 * (QSS_NSLOT - 1))
#define QSS_SPREAD (QSS_NSLOT == 2 && QSS_RLAST <= 16)
#define QSS_R2 (QSS_RLAST <= 1 ? 1 : QSS_RLAST <= 2 ? 2 : QSS_RLAST <= 4 ? 4 : QSS_RLAST <= 8 ? 8 : 16)
#define QSS_G (32 / QSS_R2)

// One pivot step k of the FP32 factorisation of qss_solve_fp32ir, on rows
// whose live part is their first W entries (the rows are shifted left one
// column per step, so from step NN - W on every entry j >= W is zero and
// stays zero): warp argmax of |A[.][0]| over the rows not yet pivoted (lowest
// row on ties), the pivot row broadcast, its U part and the multipliers
// stored to LU, and the elimination fused with the shift.  Returns false on
// a zero, infinite or NaN pivot.
template <int W>
__device__ __forceinline__ bool qss_lu32_step(const int k, float (&A)[QSS_NSLOT][QSS_NN], int (&ord)[QSS_NSLOT],
                                              const bool (&live)[QSS_NSLOT], float* __restrict__ LU,
                                              int* __restrict__ piv, float* __restrict__ pinv, const int lane) {
  int best = -1, brow = QSS_NN;
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) {
    const int key = (live[sl] && ord[sl] < 0) ? (__float_as_int(A[sl][0]) & 0x7fffffff) : -1;
    if (key > best) { best = key; brow = lane + 32 * sl; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int orow = __shfl_xor_sync(0xffffffffu, brow, off);
    if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
  }
  if (best <= 0 || best >= 0x7f800000) return false;   // zero, inf or NaN pivot
  const int pl = brow & 31, ps = brow >> 5;
  float p[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    float v = A[0][j];
#pragma unroll
    for (int sl = 1; sl < QSS_NSLOT; ++sl)
      if (ps == sl) v = A[sl][j];
    p[j] = __shfl_sync(0xffffffffu, v, pl);
  }
  const float inv = 1.0f / p[0];
  if (lane == 0) { piv[k] = brow; pinv[k] = inv; }
  if (lane == pl) {   // the pivot row's U part, columns k..NN-1
#pragma unroll
    for (int j = 0; j < W; ++j)
      if (j < QSS_NN - k) LU[brow * QSS_MSTRIDE + k + j] = p[j];
  }
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl)
    if (lane == pl && ps == sl) ord[sl] = k;
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) {
    const bool el = live[sl] && ord[sl] < 0;
    const float l = el ? A[sl][0] * inv : 0.0f;
    if (el) LU[(lane + 32 * sl) * QSS_MSTRIDE + k] = l;
#pragma unroll
    for (int j = 0; j + 1 < W; ++j) A[sl][j] = fmaf(-l, p[j + 1], A[sl][j + 1]);
    A[sl][W - 1] = 0.0f;
  }
  return true;
}

// FP32 LU with FP64 iterative refinement of one cell's Newton system
// (I - h J) x = g.  J (FP64) is in shared memory, row r at Js[r * QSS_MSTRIDE];
// the warp's lanes own rows lane + 32 slot.
//   Equilibration: row exponents er_r and column exponents ec_j (powers of
//   two, from the exponent fields of h and J: every scaled entry of
//   I - h J is below 4 in magnitude), so that FP32 holds every entry near 1.
//   The scaled FP32 matrix is built in registers from J's bits: h J_rj 2^-s
//   = hm * float(J_rj 2^(eh - s)) with h = hm 2^eh, plus 2^-s on the diagonal
//   (integer and FP32 operations only).
//   Factorisation: compact by design (an unrolled FP32 elimination is
//   fetch-bound): loops over pivot steps with the live rows in registers
//   shifted left by one column per step (the pivot column is always entry 0,
//   the shift folds into the elimination FMA), in four phases of decreasing
//   static width (qss_lu32_step); L and U go to shared memory
//   (LU[r][k]: multiplier of row r at step k before its pivot step, its U row
//   from there on), and the substitutions are loops over them.
//   Refinement: r = g - x + h (J x) in FP64 (the rows of a thin last slot
//   spread over the warp), scaled to FP32 by powers of two, corrected through
//   the FP32 factors, until the correction is below refine_tol relative (or
//   the next one, extrapolated from the observed contraction, is below a
//   tenth of it), stops shrinking, or after max_refine sweeps.
// Returns false on a zero or non-finite FP32 pivot, or when a refinement
// sweep produces a non-finite correction (the caller then solves the cell in
// FP64).
__device__ __forceinline__ bool qss_solve_fp32ir(const double* __restrict__ Js, const double h,
                                                 float* __restrict__ LU, int* __restrict__ se,
                                                 int* __restrict__ piv, float* __restrict__ pinv,
                                                 double* __restrict__ sx, const double (&gr)[QSS_NSLOT],
                                                 double (&xo)[QSS_NSLOT], const int lane,
                                                 const QssNewtonOpts& o) {
  const int eh = qss_ilogb(h);
  const float hm = qss_scaled_float(h, eh);   // h's mantissa, in [1, 2)
  int er[QSS_NSLOT];
  bool live[QSS_NSLOT];
  // row exponents: er_r >= eh + e(J_rj) + 1 for every j, and >= 0 (the 1 on
  // the diagonal)
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) {
    const int r = lane + 32 * sl;
    live[sl] = r < QSS_NN;
    int mx = 0;
    if (live[sl]) {
#pragma unroll 4
      for (int j = 0; j < QSS_NN; ++j) {
        const int ej = (__double2hiint(Js[r * QSS_MSTRIDE + j]) >> 20) & 0x7ff;
        if (ej != 0) mx = max(mx, ej - 1023 + eh + 1);
      }
      se[r] = mx;
    }
    er[sl] = mx;
  }
  __syncwarp();
  // column exponents (a lane per column): ec_j >= eh + e(J_rj) + 1 - er_r,
  // and >= -er_j (the diagonal's 1)
  int ec[QSS_NSLOT];
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) {
    const int c = lane + 32 * sl;
    ec[sl] = 0;
    if (c < QSS_NN) {
      int em = -se[c];
#pragma unroll 4
      for (int r = 0; r < QSS_NN; ++r) {
        const int ej = (__double2hiint(Js[r * QSS_MSTRIDE + c]) >> 20) & 0x7ff;
        if (ej != 0) em = max(em, ej - 1023 + eh + 1 - se[r]);
      }
      ec[sl] = em;
      se[QSS_NN + c] = em;
    }
  }
  __syncwarp();
  // the scaled FP32 matrix, this lane's rows, in registers
  float A[QSS_NSLOT][QSS_NN];
  int ord[QSS_NSLOT];
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) {
    const int r = lane + 32 * sl;
    ord[sl] = -1;
#pragma unroll
    for (int j = 0; j < QSS_NN; ++j) {
      float v = 0.0f;
      if (live[sl]) {
        const int sc = er[sl] + se[QSS_NN + j];
        const float jf = qss_scaled_float(Js[r * QSS_MSTRIDE + j], sc - eh);
        v = fmaf(-hm, jf, r == j ? qss_pow2f_neg(sc) : 0.0f);
      }
      A[sl][j] = v;
    }
  }
  // factorisation, one pivot step per iteration, in four phases whose
  // static width is the live part of the shifted rows (NN - k0 columns from
  // pivot step k0 on): 2.5/4 of the full-width work for NN = 36
  constexpr int K1 = (QSS_NN + 3) / 4, K2 = (2 * QSS_NN + 3) / 4, K3 = (3 * QSS_NN + 3) / 4;
#pragma unroll 1
  for (int k = 0; k < K1; ++k)
    if (!qss_lu32_step<QSS_NN>(k, A, ord, live, LU, piv, pinv, lane)) return false;
#pragma unroll 1
  for (int k = K1; k < K2; ++k)
    if (!qss_lu32_step<QSS_NN - K1>(k, A, ord, live, LU, piv, pinv, lane)) return false;
#pragma unroll 1
  for (int k = K2; k < K3; ++k)
    if (!qss_lu32_step<QSS_NN - K2>(k, A, ord, live, LU, piv, pinv, lane)) return false;
#pragma unroll 1
  for (int k = K3; k < QSS_NN; ++k)
    if (!qss_lu32_step<QSS_NN - K3>(k, A, ord, live, LU, piv, pinv, lane)) return false;
  __syncwarp();
  // refinement: r = g - x + h (J x) in FP64, correction from the FP32 factors
#pragma unroll
  for (int sl = 0; sl < QSS_NSLOT; ++sl) xo[sl] = 0.0;
  double prev = 1e308;
#pragma unroll 1
  for (int sweep = 0; sweep <= o.max_refine; ++sweep) {
    double res[QSS_NSLOT];
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) res[sl] = live[sl] ? gr[sl] : 0.0;
    if (sweep > 0) {
      double jx[QSS_NSLOT];
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl) {
        jx[sl] = 0.0;
        if (QSS_SPREAD && sl == QSS_NSLOT - 1) continue;
        if (live[sl]) {
          const int r = lane + 32 * sl;
          double acc = 0.0;
#pragma unroll 6
          for (int j = 0; j < QSS_NN; ++j) acc = fma(Js[r * QSS_MSTRIDE + j], sx[j], acc);
          jx[sl] = acc;
        }
      }
      if (QSS_SPREAD) {
        // rows 32.. of the thin last slot: lane l takes row 32 + (l mod R2)
        // and columns l / R2 + G m; the partial sums of a row meet in its
        // lane l < R by a butterfly over the lanes of equal l mod R2
        const int rr = lane & (QSS_R2 - 1);
        const int r = 32 + rr;
        double acc = 0.0;
        if (rr < QSS_RLAST) {
#pragma unroll
          for (int m = 0; m < (QSS_NN + QSS_G - 1) / QSS_G; ++m) {
            const int j = lane / QSS_R2 + QSS_G * m;
            if (j < QSS_NN) acc = fma(Js[r * QSS_MSTRIDE + j], sx[j], acc);
          }
        }
#pragma unroll
        for (int off = QSS_R2; off < 32; off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        jx[QSS_NSLOT - 1] = acc;
      }
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl)
        if (live[sl]) res[sl] = fma(h, jx[sl], res[sl] - xo[sl]);
    }
    // scale to FP32: z_r = res_r 2^-(er_r + es), es the largest row exponent
    int emax = -4000;
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) {
      const int eb = (__double2hiint(res[sl]) >> 20) & 0x7ff;
      if (live[sl] && eb != 0) emax = max(emax, eb - 1023 - er[sl]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    if (emax == -4000) break;   // zero residual: x is exact
    const int es = emax;
    float z[QSS_NSLOT];
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) z[sl] = live[sl] ? qss_scaled_float(res[sl], er[sl] + es) : 0.0f;
    // forward substitution
#pragma unroll 1
    for (int k = 0; k < QSS_NN; ++k) {
      const int pr = piv[k];
      const int pl = pr & 31, ps = pr >> 5;
      float v = z[0];
#pragma unroll
      for (int sl = 1; sl < QSS_NSLOT; ++sl)
        if (ps == sl) v = z[sl];
      const float zp = __shfl_sync(0xffffffffu, v, pl);
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl)
        if (live[sl] && ord[sl] > k) z[sl] = fmaf(-LU[(lane + 32 * sl) * QSS_MSTRIDE + k], zp, z[sl]);
    }
    // back substitution, column oriented: lane (k & 31) keeps x_k
    float d[QSS_NSLOT];
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) d[sl] = 0.0f;
#pragma unroll 1
    for (int k = QSS_NN - 1; k >= 0; --k) {
      const int pr = piv[k];
      const int pl = pr & 31, ps = pr >> 5;
      float v = z[0];
#pragma unroll
      for (int sl = 1; sl < QSS_NSLOT; ++sl)
        if (ps == sl) v = z[sl];
      const float xk = __shfl_sync(0xffffffffu, v, pl) * pinv[k];
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl)
        if (lane == (k & 31) && (k >> 5) == sl) d[sl] = xk;
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl)
        if (live[sl] && ord[sl] < k) z[sl] = fmaf(-LU[(lane + 32 * sl) * QSS_MSTRIDE + k], xk, z[sl]);
    }
    // correction dd_j = d_j 2^(es - ec_j), x += dd
    long long dmx = 0, xmx = 0;
    bool dfin = true;
    __syncwarp();
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) {
      const int j = lane + 32 * sl;
      if (j < QSS_NN) {
        dfin = dfin && (__float_as_uint(d[sl]) & 0x7f800000u) != 0x7f800000u;
        const double dd = qss_float_to_double_scaled(d[sl], es - ec[sl]);
        xo[sl] += dd;
        sx[j] = xo[sl];
        dmx = max(dmx, qss_absbits(dd));
        xmx = max(xmx, qss_absbits(xo[sl]));
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      dmx = max(dmx, __shfl_xor_sync(0xffffffffu, dmx, off));
      xmx = max(xmx, __shfl_xor_sync(0xffffffffu, xmx, off));
    }
    if (!__all_sync(0xffffffffu, dfin) || dmx >= 0x7ff0000000000000LL || xmx >= 0x7ff0000000000000LL)
      return false;
    __syncwarp();
    const double dmax = __longlong_as_double(dmx), xmax = __longlong_as_double(xmx);
    if (dmax <= o.refine_tol * xmax || dmax >= 0.5 * prev) break;
    // the next correction, extrapolated from this sweep's contraction
    // dmax / prev, is below a tenth of the target: the current x is already
    // that accurate, so the sweep that would confirm it is skipped
    if (sweep > 0 && dmax * dmax <= 0.1 * o.refine_tol * xmax * prev) break;
    prev = dmax;
  }
  return true;
}

// Jacobian reuse (opt-in, qss_newton_opts.jac_reuse): the squared weighted
// norm of a cell's Newton update must shrink by this factor from one
// iteration to the next (the norm by 0.3) for the kept Jacobian to be used
// again; otherwise the next iteration evaluates a fresh one.
#define QSS_REUSE_RATE2 0.09

// mode 0: full Newton (J fresh every iteration, at list position t of M64;
//         the next iteration's list is LIST2);
// mode 1: J fresh at M64[t], copied to the cell's slot of JK (JK[s * NNZ +
//         e]) for later iterations; the cell continues on LIST3 (f only);
// mode 2: J from JK (kept); the cell continues on LIST3 while its update
//         norm contracts by QSS_REUSE_RATE2 (squared), else on LIST2 (fresh
//         J); an update whose norm grew, or that is not finite, is not
//         applied (the cell retries from the same state with a fresh J).
//         DN[s] holds the previous iteration's squared norm.
template <bool FP32IR>
__device__ __forceinline__ void qss_newton_update(
    long long c0, const double* __restrict__ dt, int dt_stride, double* __restrict__ PHI,
    const double* __restrict__ PHI0, const double* __restrict__ F, const double* __restrict__ M64,
    int* __restrict__ ACT, int* __restrict__ ST, int* __restrict__ IT, const int* __restrict__ LIST,
    const int* __restrict__ NACT, int* __restrict__ LIST2, int* __restrict__ NACT2, long long sld,
    double* __restrict__ FN0, double* __restrict__ FN1, const QssNewtonOpts o, const int mode,
    double* __restrict__ JK, double* __restrict__ DN, int* __restrict__ LIST3, int* __restrict__ NACT3) {
  constexpr int W = FP32IR ? QSS_UPD_WARPS32 : QSS_UPD_WARPS;
  const unsigned FULL = 0xffffffffu;
  // per-warp copy of the FP64 Newton matrix M = I - dt J (padded rows; the
  // FP64 form keeps g in the pad column and solves in place)
  __shared__ double sh_m[W * QSS_NN * QSS_MSTRIDE];
  // FP32_IR: pivot order, solution, the FP32 factors, scale exponents and
  // pivot reciprocals
  __shared__ int sh_piv[FP32IR ? W : 1][QSS_NN];
  __shared__ double sh_x[FP32IR ? W : 1][QSS_NN + 1];
  __shared__ float sh_lu[FP32IR ? W * QSS_NN * QSS_MSTRIDE : 1];
  __shared__ int sh_e[FP32IR ? W : 1][2 * QSS_NN];
  __shared__ float sh_pinvf[FP32IR ? W : 1][QSS_NN];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nact = *NACT;
  QSS_DBG_CHECK(nact >= 0 && nact <= sld, 6);
  const long long nwarps = (long long)gridDim.x * W;
  double* Ms = &sh_m[w * QSS_NN * QSS_MSTRIDE];   // this warp's copy of [M | g], M = I - h J
  // one active cell per warp at a time, the warps striding over the list:
  // when few cells are left (the last Newton iterations) each gets its own
  // warp instead of queueing behind 31 others
  for (long long tq = (long long)blockIdx.x * W + w; tq < nact; tq += nwarps) {
    const int s = LIST[tq];
    QSS_DBG_CHECK(s >= 0 && s < sld, 7);   // warp-uniform: the whole warp leaves
    const double hq = dt[dt_stride ? c0 + s : 0];
    const int it = IT[s] + 1;
    // g = -G(phi) = -(phi - phi0 - h f), entry i on lane i % 32 (slot i / 32);
    // f optionally recorded at the first iterate (phi0) and the latest
    double gr[QSS_NSLOT];
    bool ok = true;
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) {
      const int i = lane + 32 * sl;
      gr[sl] = 0.0;
      if (i < QSS_NN) {
        const double f = F[i * sld + tq];
        if (FN0 && it == 1) FN0[i * sld + s] = f;
        if (FN1) FN1[i * sld + s] = f;
        gr[sl] = -(PHI[i * sld + s] - PHI0[i * sld + s] - hq * f);
        ok = ok && qss_finite(gr[sl]);
      }
    }
    __syncwarp();
    if (lane == 0) IT[s] = it;
    if (!__all_sync(FULL, ok)) {
      if (lane == 0) { ST[s] = QSS_CELL_NONFINITE; ACT[s] = 0; }
      continue;
    }
    bool fin = true;
    {
      // the cell's J, interleaved with three neighbours (the Jacobian
      // kernel's list-mode layout): every 32-byte sector this warp loads also
      // holds the same entry of the cells the next warps take
      const double* __restrict__ Jq = mode == 2 ? JK + (long long)s * QSS_JAC_NNZ
                                                : M64 + (tq >> 2) * (4 * QSS_JAC_NNZ) + (tq & 3);
      const int js = mode == 2 ? 1 : 4;   // element stride of that J
      double* __restrict__ Jk = mode == 1 ? JK + (long long)s * QSS_JAC_NNZ : nullptr;
#ifdef QSS_JAC_CSR
      // CSR values: M = I first, then M[i][j] += -h J_ij at the stored
      // positions (each position once; 1 + m and 0 + m round as the dense
      // form's 1 + m and m)
      for (int e = lane; e < QSS_NN * QSS_MSTRIDE; e += 32) {
        const int r = e / QSS_MSTRIDE;
        Ms[e] = (e == r * (QSS_MSTRIDE + 1) && !FP32IR) ? 1.0 : 0.0;
      }
      __syncwarp();
      const int eh = qss_ilogb(hq);
#pragma unroll 4
      for (int p = lane; p < QSS_JAC_NNZ; p += 32) {
        const int rc = qss_jac_rc[p];
        const int r = rc / QSS_NN, j = rc - r * QSS_NN;
        const double v = Jq[js * p];
        if (Jk) Jk[p] = v;
        if constexpr (FP32IR) {   // J itself (see the dense branch)
          fin = fin && qss_finite(v) && qss_ilogb(v) + eh < 1020;
          Ms[r * QSS_MSTRIDE + j] = v;
        } else {
          const double m = -hq * v;
          fin = fin && qss_finite(m);
          Ms[r * QSS_MSTRIDE + j] += m;
        }
      }
#else
      if constexpr (FP32IR) {
        // J itself (no FP64 operation): the FP32-IR solve builds its scaled
        // FP32 matrix from J's bits and forms the residual from J; h J must
        // not overflow
        const int eh = qss_ilogb(hq);
#pragma unroll 4
        for (int e = lane; e < QSS_NN * QSS_NN; e += 32) {
          const int r = e / QSS_NN, j = e - r * QSS_NN;
          const double v = Jq[js * e];
          if (Jk) Jk[e] = v;
          fin = fin && qss_finite(v) && qss_ilogb(v) + eh < 1020;
          Ms[r * QSS_MSTRIDE + j] = v;
        }
      } else {
#pragma unroll 4
        for (int e = lane; e < QSS_NN * QSS_NN; e += 32) {
          const int r = e / QSS_NN, j = e - r * QSS_NN;
          const double v = Jq[js * e];
          if (Jk) Jk[e] = v;
          const double m = -hq * v;
          fin = fin && qss_finite(m);
          Ms[r * QSS_MSTRIDE + j] = (r == j) ? 1.0 + m : m;
        }
      }
#endif
    }
    if (!FP32IR) {
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl) {
        const int r = lane + 32 * sl;
        if (r < QSS_NN) Ms[r * QSS_MSTRIDE + QSS_NN] = gr[sl];
      }
    }
    __syncwarp();
    if (!__all_sync(FULL, fin)) {
      if (lane == 0) { ST[s] = QSS_CELL_NONFINITE; ACT[s] = 0; }
      continue;
    }
    double xo[QSS_NSLOT];   // this lane's entries of the solution (index lane + 32 slot)
    bool solved;
    if constexpr (FP32IR) {
      solved = qss_solve_fp32ir(Ms, hq, &sh_lu[w * QSS_NN * QSS_MSTRIDE], sh_e[w], sh_piv[w], sh_pinvf[w],
                                sh_x[w], gr, xo, lane, o);
      if (!solved) {
        // the FP32 factorisation met a zero or non-finite pivot (or the
        // refinement diverged): solve this cell's system in FP64 instead,
        // M = I - h J formed from the intact FP64 copy of J as the FP64 form
        // forms it, so that the mixed form reports no status the FP64 form
        // would not
        __syncwarp();
        for (int e = lane; e < QSS_NN * QSS_NN; e += 32) {
          const int r = e / QSS_NN, j = e - r * QSS_NN;
          const double m = -hq * Ms[r * QSS_MSTRIDE + j];
          Ms[r * QSS_MSTRIDE + j] = (r == j) ? 1.0 + m : m;
        }
        __syncwarp();
#pragma unroll
        for (int sl = 0; sl < QSS_NSLOT; ++sl) {
          const int r = lane + 32 * sl;
          if (r < QSS_NN) Ms[r * QSS_MSTRIDE + QSS_NN] = gr[sl];
        }
        __syncwarp();
        solved = qss_smem_solve_fp64(Ms, lane);
#pragma unroll
        for (int sl = 0; sl < QSS_NSLOT; ++sl) {
          const int r = lane + 32 * sl;
          xo[sl] = r < QSS_NN ? Ms[r * QSS_MSTRIDE + QSS_NN] : 0.0;
        }
      }
    } else {
      solved = qss_smem_solve_fp64(Ms, lane);
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl) {
        const int r = lane + 32 * sl;
        xo[sl] = r < QSS_NN ? Ms[r * QSS_MSTRIDE + QSS_NN] : 0.0;
      }
    }
    __syncwarp();   // the next cell overwrites this warp's shared arrays
    if (!solved) {
      if (lane == 0) { ST[s] = QSS_CELL_SINGULAR; ACT[s] = 0; }
      continue;
    }
    // phi + x and the weighted RMS of the update over the lanes; a kept-J
    // update whose norm grew (or that turned non-finite) is discarded: the
    // cell retries from the same state with a fresh Jacobian
    double acc = 0.0, pv[QSS_NSLOT];
    bool pfin = true;
#pragma unroll
    for (int sl = 0; sl < QSS_NSLOT; ++sl) {
      const int i = lane + 32 * sl;
      pv[sl] = 0.0;
      if (i < QSS_NN) {
        const double x = xo[sl];
        const double p = PHI[i * sld + s] + x;
        pv[sl] = p;
        const double wgt = o.rtol * fabs(p) + (i < QSS_N ? o.atol_C : o.atol_T);
        const double qv = x / wgt;
        acc = fma(qv, qv, acc);
        pfin = pfin && qss_finite(p);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    pfin = __all_sync(FULL, pfin);
    const bool reject = mode == 2 && !(pfin && acc <= DN[s]);
    if (!reject) {
#pragma unroll
      for (int sl = 0; sl < QSS_NSLOT; ++sl) {
        const int i = lane + 32 * sl;
        if (i < QSS_NN) PHI[i * sld + s] = pv[sl];
      }
    }
    if (lane == 0) {
      if (reject) {
        if (it >= o.max_iter) ACT[s] = 0;          // status stays MAXITER
        else LIST2[atomicAdd(NACT2, 1)] = s;       // fresh J at the same state
      } else if (!pfin) {
        ST[s] = QSS_CELL_NONFINITE;
        ACT[s] = 0;
      } else if (acc <= (double)QSS_NN) {
        ST[s] = QSS_CELL_CONVERGED;
        ACT[s] = 0;
      } else if (it >= o.max_iter) {
        ACT[s] = 0;   // status stays MAXITER
      } else if (mode == 0 || (mode == 2 && acc > QSS_REUSE_RATE2 * DN[s])) {
        LIST2[atomicAdd(NACT2, 1)] = s;   // fresh J next iteration
      } else {
        DN[s] = acc;
        LIST3[atomicAdd(NACT3, 1)] = s;   // keep J, evaluate f only
      }
    }
  }
}

#define QSS_UPDATE_PARAMS                                                                         \
  long long c0, const double* __restrict__ dt, int dt_stride, double* __restrict__ PHI,          \
      const double* __restrict__ PHI0, const double* __restrict__ F, const double* __restrict__ M64, \
      int* __restrict__ ACT, int* __restrict__ ST, int* __restrict__ IT,                          \
      const int* __restrict__ LIST, const int* __restrict__ NACT, int* __restrict__ LIST2,        \
      int* __restrict__ NACT2, long long sld, double* __restrict__ FN0, double* __restrict__ FN1, \
      QssNewtonOpts o, int mode, double* __restrict__ JK, double* __restrict__ DN,                \
      int* __restrict__ LIST3, int* __restrict__ NACT3

extern "C" __global__ void __launch_bounds__(QSS_UPD_WARPS * 32)
qss_newton_update_fp64_kernel(QSS_UPDATE_PARAMS) {
  qss_newton_update<false>(c0, dt, dt_stride, PHI, PHI0, F, M64, ACT, ST, IT, LIST, NACT, LIST2,
                           NACT2, sld, FN0, FN1, o, mode, JK, DN, LIST3, NACT3);
}

extern "C" __global__ void __launch_bounds__(QSS_UPD_WARPS32 * 32)
qss_newton_update_fp32ir_kernel(QSS_UPDATE_PARAMS) {
  qss_newton_update<true>(c0, dt, dt_stride, PHI, PHI0, F, M64, ACT, ST, IT, LIST, NACT, LIST2,
                          NACT2, sld, FN0, FN1, o, mode, JK, DN, LIST3, NACT3);
}

// Write the state back: T, Y (rho fixed), iterations and status.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_newton_finish_kernel(long long cells, long long c0, long long ld, const double* __restrict__ rho,
                         double* __restrict__ T, double* __restrict__ Y, const double* __restrict__ PHI,
                         const int* __restrict__ ST, const int* __restrict__ IT, int* __restrict__ iters,
                         int* __restrict__ status, long long sld, const int* __restrict__ ncap) {
  if (ncap) cells = min(cells, (long long)*ncap);
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  QSS_DBG_CHECK(cells <= sld, 4);
  if (s >= cells) return;
  const long long c = c0 + s;
  QSS_DBG_CHECK(c < ld, 5);
  const double r = rho[c];
  T[c] = PHI[QSS_N * sld + s];
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) Y[k * ld + c] = PHI[k * sld + s] / (r * qss_inv_W[k]);
  if (iters) iters[c] = IT[s];
  if (status) status[c] = ST[s];
}

// ---------------------------------------------------------------------------
// Integration over an interval by substeps with local error control
// (qss_integrate), backward Euler (order 1) or variable-step BDF2 (order 2,
// after a first backward-Euler substep).  Per cell s of a chunk (persistent
// across rounds):
//   TT[s] time done, HH[s] next substep, DT[s] target interval,
//   IS[s] 0 done / 1 active / 2 substep below h_min, NS[s] accepted substeps,
//   order 2: HP[s] previous accepted substep (0: none yet), PP[k S + s] and
//   FP[k S + s] the state and f at its start (phi_n-1, f_n-1).
// A round: gather the active cells (list A, count *CA) into a contiguous
// batch (rho, T, Y, Newton step gamma, constant term PC of G), one
// Newton-solved substep of the batch (f recorded at phi_n and at the last
// iterate), then accept or reject each cell's substep and build the next
// active list (B).  With w = h / h_prev, BDF2 solves
//   phi - a1 phi_n - a2 phi_n-1 - beta h f(phi) = 0,
//   a1 = (1+w)^2/(1+2w), a2 = -w^2/(1+2w), beta = (1+w)/(1+2w),
// and estimates its local error as h (1+w)/(3(1+2w)) ((f_n+1 - f_n) -
// w (f_n - f_n-1)) (its truncation error with the third derivative from the
// second divided difference of f); backward Euler's estimate is
// h/2 (f_n+1 - f_n).
struct QssIntegOpts {
  double rtol, atol_C, atol_T;
  double h_min;   // fraction of the interval
  int order;      // 1 or 2
};

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_integ_init_kernel(long long cells, long long c0, const double* __restrict__ dt_total,
                      int dt_stride, double h0, double* __restrict__ TT, double* __restrict__ HH,
                      double* __restrict__ DT, int* __restrict__ IS, int* __restrict__ NS,
                      int* __restrict__ LA, int* __restrict__ CA, double* __restrict__ HP) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s == 0) *CA = (int)cells;
  if (s >= cells) return;
  const double D = dt_total[dt_stride ? c0 + s : 0];
  DT[s] = D;
  TT[s] = 0.0;
  HH[s] = fmin(h0 > 0.0 ? h0 : 0.01 * D, D);
  HP[s] = 0.0;
  IS[s] = 1;
  NS[s] = 0;
  LA[s] = (int)s;
}

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_integ_gather_kernel(long long c0, long long ld, const double* __restrict__ rho,
                        const double* __restrict__ T, const double* __restrict__ Y,
                        const int* __restrict__ LA, const int* __restrict__ CA, int* __restrict__ CB,
                        const double* __restrict__ HH, double* __restrict__ rhob,
                        double* __restrict__ Tb, double* __restrict__ Yb, double* __restrict__ dtb,
                        int* __restrict__ ncap, long long bld, const double* __restrict__ HP,
                        const double* __restrict__ PP, double* __restrict__ PC, long long S, int order) {
  const long long i = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  const int n = *CA;
  if (i == 0) { *CB = 0; *ncap = n; }
  if (i >= n) return;
  const int s = LA[i];
  const long long c = c0 + s;
  const double r = rho[c];
  rhob[i] = r;
  Tb[i] = T[c];
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) Yb[k * bld + i] = Y[k * ld + c];
  const double h = HH[s];
  dtb[i] = h;
  if (order == 2) {
    // the constant term of G: phi_n (backward Euler) or the BDF2 combination
    const double hp = HP[s];
    double a1 = 1.0, a2 = 0.0;
    if (hp > 0.0) {
      const double w = h / hp;
      a1 = (1.0 + w) * (1.0 + w) / (1.0 + 2.0 * w);
      a2 = -w * w / (1.0 + 2.0 * w);
      dtb[i] = (1.0 + w) / (1.0 + 2.0 * w) * h;
    }
#pragma unroll
    for (int k = 0; k < QSS_NN; ++k) {
      const double phi = k < QSS_N ? r * Y[k * ld + c] * qss_inv_W[k] : T[c];
      PC[k * bld + i] = hp > 0.0 ? a1 * phi + a2 * PP[k * S + s] : phi;
    }
  }
}

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_integ_accept_kernel(long long c0, long long ld, double* __restrict__ T, double* __restrict__ Y,
                        const int* __restrict__ LA, const int* __restrict__ CA, int* __restrict__ LB,
                        int* __restrict__ CB, double* __restrict__ HH, double* __restrict__ TT,
                        const double* __restrict__ DT, int* __restrict__ IS, int* __restrict__ NS,
                        const double* __restrict__ rhob, const double* __restrict__ Tb,
                        const double* __restrict__ Yb, const int* __restrict__ bst,
                        const double* __restrict__ FN0, const double* __restrict__ FN1, long long bld,
                        QssIntegOpts o, double* __restrict__ HP, double* __restrict__ PP,
                        double* __restrict__ FP, long long S) {
  const long long i = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (i >= *CA) return;
  const int s = LA[i];
  const long long c = c0 + s;
  const double h = HH[s];
  const double g_max = o.order == 2 ? 2.0 : 4.0;
  bool keep = true;
  if (bst[i] != QSS_CELL_CONVERGED) {
    // the Newton solve failed: a quarter of the substep
    HH[s] = 0.25 * h;
  } else {
    const bool bdf2 = o.order == 2 && HP[s] > 0.0;
    const double w = bdf2 ? h / HP[s] : 0.0;
    const double ce = bdf2 ? h * (1.0 + w) / (3.0 * (1.0 + 2.0 * w)) : 0.5 * h;
    // local error estimate, weighted RMS
    const double r = rhob[i];
    double e2 = 0.0;
#pragma unroll
    for (int k = 0; k < QSS_NN; ++k) {
      const double phi = k < QSS_N ? r * Yb[k * bld + i] * qss_inv_W[k] : Tb[i];
      const double f0 = FN0[k * bld + i], f1 = FN1[k * bld + i];
      const double e = bdf2 ? ce * ((f1 - f0) - w * (f0 - FP[k * S + s])) : ce * (f1 - f0);
      const double wt = o.rtol * fabs(phi) + (k < QSS_N ? o.atol_C : o.atol_T);
      const double q = e / wt;
      e2 = fma(q, q, e2);
    }
    const double err = sqrt(e2 / QSS_NN);
    // 0.9 err^(-1/(p+1)) for the substep's order p
    const double gr = err > 0.0 ? (bdf2 ? 0.9 / cbrt(err) : 0.9 / sqrt(err)) : 0.0;
    if (err <= 1.0) {
      if (o.order == 2) {   // history for the next substep: phi_n, f_n, h
#pragma unroll
        for (int k = 0; k < QSS_NN; ++k) {
          PP[k * S + s] = k < QSS_N ? r * Y[k * ld + c] * qss_inv_W[k] : T[c];
          FP[k * S + s] = FN0[k * bld + i];
        }
        HP[s] = h;
      }
      T[c] = Tb[i];
#pragma unroll
      for (int k = 0; k < QSS_N; ++k) Y[k * ld + c] = Yb[k * bld + i];
      TT[s] += h;
      NS[s] += 1;
      const double rem = DT[s] - TT[s];
      if (rem <= 1e-12 * DT[s]) {
        IS[s] = 0;
        keep = false;
      } else {
        const double g = err > 0.0 ? gr : g_max;
        HH[s] = fmin(h * fmin(g_max, fmax(0.2, g)), rem);
      }
    } else {
      // rejected (also for a NaN error)
      const double g = err > 0.0 ? gr : 0.25;
      HH[s] = h * (g == g ? fmin(0.9, fmax(0.2, g)) : 0.25);
    }
  }
  if (keep && HH[s] < o.h_min * DT[s]) {
    IS[s] = 2;
    keep = false;
  }
  if (keep) LB[atomicAdd(CB, 1)] = s;
}

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_integ_finish_kernel(long long cells, long long c0, const int* __restrict__ IS,
                        const int* __restrict__ NS, int* __restrict__ nsteps, int* __restrict__ status) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s >= cells) return;
  const long long c = c0 + s;
  if (nsteps) nsteps[c] = NS[s];
  // 0 reached the end, 1 substep attempts exhausted, 2 substep below h_min
  if (status) status[c] = IS[s] == 0 ? 0 : (IS[s] == 2 ? 2 : 1);
}

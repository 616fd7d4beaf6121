// Implicit (backward-Euler) step kernels around a generated mechanism body.
//
// Newton on G(phi) = phi - phi0 - dt f(phi), phi = (C, T), f = (wdot, Tdot) at
// constant volume, with the matrix M = I - dt J where J is the analytic
// Jacobian, re-evaluated every iteration.  One Newton iteration is two
// launches, one thread per cell:
//   qss_jac_kernel (phi mode)        f and J at the current iterate
//   qss_newton_update_*_kernel       M = I - dt J, factor, solve, update phi,
//                                    convergence test
// so that the long generated body is compiled once (in qss_jac_kernel) and the
// linear algebra runs at its own occupancy.  Cells that have converged (or
// failed) are inactive and return at once in both kernels; the host enqueues
// max_iter iterations without synchronising.
//   update_fp64    LU of M with partial pivoting in FP64.
//   update_fp32ir  M equilibrated by powers of two (rows, then columns), LU
//                  with partial pivoting in FP32, the solution refined with
//                  FP64 residuals b - M x until the correction is below
//                  refine_tol relative or max_refine sweeps.
// Rates, equilibrium constants, the QSS solve, J, M and the Newton residual
// are FP64 in both forms.
//
// Scratch (global memory, structure of arrays with leading dimension sld, for
// one chunk of cells, s = c - c0):
//   M64[e * sld + s], e = i * NN + j   J, then the FP64 Newton matrix / factors
//   M32[e * sld + s]                   the FP32 factors (FP32_IR only)
//   PHI, PHI0, F [k * sld + s]         iterate, initial state, f
//   ACT, ST, IT [s]                    active flag, status, iteration count
// Every access of a warp to one entry is one contiguous segment; only the row
// swaps of pivoting touch different rows per thread.
#pragma once

#define QSS_CELL_CONVERGED 0
#define QSS_CELL_MAXITER 1
#define QSS_CELL_NONFINITE 2
#define QSS_CELL_SINGULAR 3

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

__device__ __forceinline__ double qss_pow2(int e) {   // 2^e, |e| <= 1022
  return __hiloint2double((e + 1023) << 20, 0);
}

// Magnitude key for pivot search: integer order of |x| for doubles (keeps the
// comparisons off the FP64 pipe), |x| itself for floats.
__device__ __forceinline__ long long qss_mag(double x) { return qss_absbits(x); }
__device__ __forceinline__ float qss_mag(float x) { return fabsf(x); }

// In-place LU with partial pivoting (physical row swaps) of an NN x NN matrix
// stored at A[e * sld], e = i * NN + j.  Returns false on a zero pivot.
template <class R>
__device__ __forceinline__ bool qss_lu(R* __restrict__ A, const long long sld, int* __restrict__ perm) {
#pragma unroll 1
  for (int k = 0; k < QSS_NN; ++k) {
    int p = k;
    auto best = qss_mag(A[(k * QSS_NN + k) * sld]);
#pragma unroll 1
    for (int i = k + 1; i < QSS_NN; ++i) {
      const auto v = qss_mag(A[(i * QSS_NN + k) * sld]);
      if (v > best) { best = v; p = i; }
    }
    perm[k] = p;
    if (!(best > 0)) return false;
    if (p != k) {
#pragma unroll 1
      for (int j = 0; j < QSS_NN; ++j) {
        const R t = A[(k * QSS_NN + j) * sld];
        A[(k * QSS_NN + j) * sld] = A[(p * QSS_NN + j) * sld];
        A[(p * QSS_NN + j) * sld] = t;
      }
    }
    const R inv = R(1) / A[(k * QSS_NN + k) * sld];
#pragma unroll 1
    for (int i = k + 1; i < QSS_NN; ++i) {
      const R l = A[(i * QSS_NN + k) * sld] * inv;
      A[(i * QSS_NN + k) * sld] = l;
      if (l != R(0)) {
#pragma unroll 4
        for (int j = k + 1; j < QSS_NN; ++j)
          A[(i * QSS_NN + j) * sld] = fma(-l, A[(k * QSS_NN + j) * sld], A[(i * QSS_NN + j) * sld]);
      }
    }
  }
  return true;
}

// Solve with the factors of qss_lu: x = M^-1 b (b permuted and overwritten).
template <class R>
__device__ __forceinline__ void qss_lu_solve(const R* __restrict__ A, const long long sld,
                                             const int* __restrict__ perm, R* __restrict__ b) {
#pragma unroll 1
  for (int k = 0; k < QSS_NN; ++k) {
    const int p = perm[k];
    if (p != k) { const R t = b[k]; b[k] = b[p]; b[p] = t; }
  }
#pragma unroll 1
  for (int i = 1; i < QSS_NN; ++i) {
    R s = b[i];
#pragma unroll 4
    for (int j = 0; j < i; ++j) s = fma(-A[(i * QSS_NN + j) * sld], b[j], s);
    b[i] = s;
  }
#pragma unroll 1
  for (int i = QSS_NN - 1; i >= 0; --i) {
    R s = b[i];
#pragma unroll 4
    for (int j = i + 1; j < QSS_NN; ++j) s = fma(-A[(i * QSS_NN + j) * sld], b[j], s);
    b[i] = s / A[(i * QSS_NN + i) * sld];
  }
}

struct QssNewtonOpts {
  int max_iter;
  double rtol, atol_C, atol_T;
  int max_refine;
  double refine_tol;
};

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_newton_setup_kernel(long long cells, long long c0, long long ld, const double* __restrict__ rho,
                        const double* __restrict__ T, const double* __restrict__ Y,
                        double* __restrict__ PHI, double* __restrict__ PHI0, int* __restrict__ ACT,
                        int* __restrict__ ST, int* __restrict__ IT, long long sld) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s >= cells) return;
  const long long c = c0 + s;
  const double r = rho[c];
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) {
    const double v = r * Y[k * ld + c] * qss_inv_W[k];
    PHI[k * sld + s] = v;
    PHI0[k * sld + s] = v;
  }
  PHI[QSS_N * sld + s] = T[c];
  PHI0[QSS_N * sld + s] = T[c];
  ACT[s] = 1;
  ST[s] = QSS_CELL_MAXITER;
  IT[s] = 0;
}

template <bool FP32IR>
__device__ __forceinline__ void qss_newton_update(const long long s, const double h,
                                                  double* __restrict__ PHI, const double* __restrict__ PHI0,
                                                  const double* __restrict__ F, double* __restrict__ M64,
                                                  float* __restrict__ M32, int* __restrict__ ACT,
                                                  int* __restrict__ ST, int* __restrict__ IT,
                                                  const long long sld, const QssNewtonOpts o) {
  double b[QSS_NN], x[QSS_NN], g[QSS_NN], f[QSS_NN];
  int perm[QSS_NN];
  IT[s] += 1;
  double* A = M64 + s;
  bool ok = true;
#pragma unroll
  for (int i = 0; i < QSS_NN; ++i) {
    b[i] = -(PHI[i * sld + s] - PHI0[i * sld + s] - h * F[i * sld + s]);
    ok = ok && qss_finite(b[i]);
  }
  // M = I - h J in place
#pragma unroll 1
  for (int e = 0; e < QSS_NN * QSS_NN; ++e) {
    const double v = -h * A[e * sld];
    A[e * sld] = (e % (QSS_NN + 1) == 0) ? 1.0 + v : v;
    ok = ok && qss_finite(v);
  }
  if (!ok) { ST[s] = QSS_CELL_NONFINITE; ACT[s] = 0; return; }
  if (!FP32IR) {
    if (!qss_lu<double>(A, sld, perm)) { ST[s] = QSS_CELL_SINGULAR; ACT[s] = 0; return; }
#pragma unroll
    for (int i = 0; i < QSS_NN; ++i) x[i] = b[i];
    qss_lu_solve<double>(A, sld, perm, x);
  } else {
    // power-of-two equilibration: rows, then columns
    int er[QSS_NN], ec[QSS_NN];
#pragma unroll 1
    for (int i = 0; i < QSS_NN; ++i) {
      long long mx = 0;
#pragma unroll 4
      for (int j = 0; j < QSS_NN; ++j) mx = max(mx, qss_absbits(A[(i * QSS_NN + j) * sld]));
      const int e = qss_ilogb(__longlong_as_double(mx));
      er[i] = e < -1000 ? 0 : e;
    }
#pragma unroll 1
    for (int j = 0; j < QSS_NN; ++j) {
      int emax = -1100;
#pragma unroll 4
      for (int i = 0; i < QSS_NN; ++i) {
        const double v = A[(i * QSS_NN + j) * sld];
        if (qss_absbits(v) != 0) emax = max(emax, qss_ilogb(v) - er[i]);
      }
      ec[j] = emax < -1000 ? 0 : emax;
    }
    float* Fm = M32 + s;
#pragma unroll 1
    for (int i = 0; i < QSS_NN; ++i) {
#pragma unroll 4
      for (int j = 0; j < QSS_NN; ++j) {
        const int e = -(er[i] + ec[j]);
        const double scaled = A[(i * QSS_NN + j) * sld] * qss_pow2(max(min(e, 1000), -1000));
        Fm[(i * QSS_NN + j) * sld] = (float)scaled;
      }
    }
    if (!qss_lu<float>(Fm, sld, perm)) { ST[s] = QSS_CELL_SINGULAR; ACT[s] = 0; return; }
    // x = D_c (LU32)^-1 D_r b, refined with FP64 residuals
    float y[QSS_NN];
#pragma unroll
    for (int i = 0; i < QSS_NN; ++i) { x[i] = 0.0; g[i] = b[i]; f[i] = b[i]; }
#pragma unroll 1
    for (int sweep = 0; sweep <= o.max_refine; ++sweep) {
      // the right-hand side is row-scaled, then normalised by a power of two
      long long rmx = 0;
#pragma unroll
      for (int i = 0; i < QSS_NN; ++i) {
        b[i] = f[i] * qss_pow2(max(min(-er[i], 1000), -1000));
        rmx = max(rmx, qss_absbits(b[i]));
      }
      const int es = max(min(qss_ilogb(__longlong_as_double(rmx)), 1000), -1000);
      const double rs = qss_pow2(-es);
#pragma unroll
      for (int i = 0; i < QSS_NN; ++i) y[i] = (float)(b[i] * rs);
      qss_lu_solve<float>(Fm, sld, perm, y);
      double dmax = 0.0, xmax = 0.0;
#pragma unroll
      for (int j = 0; j < QSS_NN; ++j) {
        const double d = (double)y[j] * qss_pow2(max(min(es - ec[j], 1000), -1000));
        x[j] += d;
        dmax = fmax(dmax, fabs(d));
        xmax = fmax(xmax, fabs(x[j]));
      }
      if (dmax <= o.refine_tol * xmax || sweep == o.max_refine) break;
      // residual f = g - M x in FP64
#pragma unroll 1
      for (int i = 0; i < QSS_NN; ++i) {
        double acc = g[i];
#pragma unroll 4
        for (int j = 0; j < QSS_NN; ++j) acc = fma(-A[(i * QSS_NN + j) * sld], x[j], acc);
        f[i] = acc;
      }
    }
  }
  double acc = 0.0;
  bool fin = true;
#pragma unroll
  for (int i = 0; i < QSS_NN; ++i) {
    const double p = PHI[i * sld + s] + x[i];
    PHI[i * sld + s] = p;
    const double w = o.rtol * fabs(p) + (i < QSS_N ? o.atol_C : o.atol_T);
    const double q = x[i] / w;
    acc = fma(q, q, acc);
    fin = fin && qss_finite(p);
  }
  if (!fin) { ST[s] = QSS_CELL_NONFINITE; ACT[s] = 0; return; }
  if (acc <= (double)QSS_NN) { ST[s] = QSS_CELL_CONVERGED; ACT[s] = 0; return; }
  if (IT[s] >= o.max_iter) ACT[s] = 0;   // status stays MAXITER
}

#define QSS_UPDATE_PARAMS                                                                        \
  long long cells, long long c0, const double* __restrict__ dt, int dt_stride,                   \
      double* __restrict__ PHI, const double* __restrict__ PHI0, const double* __restrict__ F,   \
      double* __restrict__ M64, float* __restrict__ M32, int* __restrict__ ACT,                  \
      int* __restrict__ ST, int* __restrict__ IT, long long sld, QssNewtonOpts o

extern "C" __global__ void __launch_bounds__(QSS_BLOCK) qss_newton_update_fp64_kernel(QSS_UPDATE_PARAMS) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s >= cells || !ACT[s]) return;
  qss_newton_update<false>(s, dt[dt_stride ? c0 + s : 0], PHI, PHI0, F, M64, M32, ACT, ST, IT, sld, o);
}

extern "C" __global__ void __launch_bounds__(QSS_BLOCK) qss_newton_update_fp32ir_kernel(QSS_UPDATE_PARAMS) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s >= cells || !ACT[s]) return;
  qss_newton_update<true>(s, dt[dt_stride ? c0 + s : 0], PHI, PHI0, F, M64, M32, ACT, ST, IT, sld, o);
}

// Write the state back: T, Y (rho fixed), iterations and status.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_newton_finish_kernel(long long cells, long long c0, long long ld, const double* __restrict__ rho,
                         double* __restrict__ T, double* __restrict__ Y, const double* __restrict__ PHI,
                         const int* __restrict__ ST, const int* __restrict__ IT, int* __restrict__ iters,
                         int* __restrict__ status, long long sld) {
  const long long s = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (s >= cells) return;
  const long long c = c0 + s;
  const double r = rho[c];
  T[c] = PHI[QSS_N * sld + s];
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) Y[k * ld + c] = PHI[k * sld + s] / (r * qss_inv_W[k]);
  if (iters) iters[c] = IT[s];
  if (status) status[c] = ST[s];
}

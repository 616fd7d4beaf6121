// Source-term kernels around a generated qss_eval_wdot (one thread per cell;
// the layout is in qss_cells.cuh): the production rates and temperature
// derivative, and a finite-difference Jacobian built from them.
#pragma once

#include "qss_cells.cuh"

extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_wdot_kernel(long long ncells, long long ld, const double* __restrict__ rho,
                const double* __restrict__ T, const double* __restrict__ Y,
                double* __restrict__ wdot, double* __restrict__ Tdot) {
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (c >= ncells) return;
  double C[QSS_N];
  qss_unpack(c, ld, rho, Y, C);
  qss_eval_wdot(C, __ldg(T + c), wdot + c, Tdot ? Tdot + c : nullptr, ld);
}

// Central finite-difference Jacobian of f = (wdot, Tdot) in phi = (C, T)
// (Section 3.2: the FD Jacobian the analytic one is measured against, Eq.
// frobErr): column j = (f(phi + h e_j) - f(phi - h e_j)) / (2 h), h = dC for
// the concentrations and dT for the temperature.  2(N + 1) evaluations of the
// source term per cell, through one inlined copy of it: f(phi + h e_j) is
// written straight into column j of jac and f(phi - h e_j) into a per-thread
// buffer, then subtracted in place.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_jac_fd_kernel(long long ncells, long long ld, const double* __restrict__ rho,
                  const double* __restrict__ T, const double* __restrict__ Y, double dC,
                  double dT, double* __restrict__ jac) {
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  if (c >= ncells) return;
  double p[QSS_NN];
  double fm[QSS_NN];
  qss_unpack(c, ld, rho, Y, p);
  p[QSS_N] = __ldg(T + c);
  const long long col = (long long)QSS_NN * ld;
#pragma unroll 1
  for (int e = 0; e < 2 * QSS_NN; ++e) {
    const int j = e >> 1;
    const bool minus = e & 1;
    const double x = p[j];
    const double h = j < QSS_N ? dC : dT;
    double* out = jac + (long long)j * ld + c;            // entry (0, j)
    p[j] = minus ? x - h : x + h;
    qss_eval_wdot(p, p[QSS_N], minus ? fm : out, minus ? fm + QSS_N : out + QSS_N * col,
                  minus ? 1 : col);
    p[j] = x;
    if (minus) {
#pragma unroll 1
      for (int i = 0; i < QSS_NN; ++i) out[i * col] = (out[i * col] - fm[i]) / (2.0 * h);
    }
  }
}

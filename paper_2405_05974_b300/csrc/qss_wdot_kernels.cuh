// Source-term kernels around a generated qss_eval_wdot (one thread per cell;
// the layout is in qss_cells.cuh): the production rates and temperature
// derivative, and a finite-difference Jacobian built from them.
#pragma once

#include "qss_cells.cuh"

// f = (wdot, Tdot) from (rho, T, Y) or, in list mode (phi and list given), of
// the t-th cell of the list: s = list[t] for t < *nact, state
// phi[k * ld + s] = (C_1..C_N, T), f written at column t (wdot[k * ld + t],
// Tdot[t]); thread 0 then also clears *nact_next (the counter the following
// Newton update fills).  List mode serves the implicit step's iterations
// that keep the previous Jacobian.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_wdot_kernel(long long ncells, long long ld, const double* __restrict__ rho,
                const double* __restrict__ T, const double* __restrict__ Y,
                double* __restrict__ wdot, double* __restrict__ Tdot, const double* __restrict__ phi,
                const int* __restrict__ list, const int* __restrict__ nact, int* __restrict__ nact_next) {
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double C[QSS_N];
  double Tc;
  if (phi) {
    if (c == 0) *nact_next = 0;
    if (c >= *nact) return;
    QSS_DBG_CHECK(*nact <= ld, 1);
    const long long s = list[c];
    QSS_DBG_CHECK(s >= 0 && s < ld, 2);
#pragma unroll
    for (int k = 0; k < QSS_N; ++k) C[k] = phi[k * ld + s];
    Tc = phi[QSS_N * ld + s];
  } else {
    if (c >= ncells) return;
    QSS_DBG_CHECK(c < ld, 3);
    qss_unpack(c, ld, rho, Y, C);
    Tc = __ldg(T + c);
  }
  qss_eval_wdot(C, Tc, wdot + c, Tdot ? Tdot + c : nullptr, ld);
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
  QSS_DBG_CHECK(c < ld, 3);
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

// Kernel templates around a generated mechanism body (one thread per cell).
//
// Layout (all FP64, structure of arrays with leading dimension ld >= ncells):
//   rho[ld], T[ld], Y[k * ld + c] (k < N), wdot[k * ld + c], Tdot[ld],
//   jac[(i * (N + 1) + j) * ld + c]  (row i = d f_i, column j = d/d phi_j,
//   phi = (C_1..C_N, T)).
// Consecutive threads take consecutive cells, so every load and store of a
// warp is one contiguous 256-byte segment.
#pragma once

#ifndef QSS_BLOCK
#define QSS_BLOCK 128
#endif

__device__ __forceinline__ void qss_unpack(long long c, long long ld, const double* __restrict__ rho,
                                           const double* __restrict__ Y, double* C) {
  const double r = __ldg(rho + c);
#pragma unroll
  for (int k = 0; k < QSS_N; ++k) C[k] = r * __ldg(Y + k * ld + c) * qss_inv_W[k];
}

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

// f = (wdot, Tdot) and J.  State from (rho, T, Y) or, in list mode (phi and
// list given), of the t-th cell of the list: s = list[t] for t < *nact, state
// phi[k * ld + s] = (C_1..C_N, T), outputs written at column t.  In list mode
// thread 0 also clears *nact_next, the counter the following Newton update
// fills.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_jac_kernel(long long ncells, long long ld, const double* __restrict__ rho,
               const double* __restrict__ T, const double* __restrict__ Y,
               double* __restrict__ jac, double* __restrict__ wdot, double* __restrict__ Tdot,
               const double* __restrict__ phi, const int* __restrict__ list,
               const int* __restrict__ nact, int* __restrict__ nact_next) {
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double C[QSS_N];
  double Tc;
  if (phi) {
    if (c == 0) *nact_next = 0;
    if (c >= *nact) return;
    const long long s = list[c];
#pragma unroll
    for (int k = 0; k < QSS_N; ++k) C[k] = phi[k * ld + s];
    Tc = phi[QSS_N * ld + s];
  } else {
    if (c >= ncells) return;
    qss_unpack(c, ld, rho, Y, C);
    Tc = __ldg(T + c);
  }
  qss_eval_jac(C, Tc, wdot ? wdot + c : nullptr, Tdot ? Tdot + c : nullptr, jac + c, ld, ld);
}

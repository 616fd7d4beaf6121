// The mixed-precision Jacobian kernel around the generated qss_eval_jac32
// (one thread per cell).  Its interface, modes and storage layouts are those
// of qss_jac_kernel: (rho, T, Y) SoA in, or list mode for the implicit step
// (state of cell list[t] from phi, f at column t, J in groups of four cells).
// wdot and Tdot are the FP64 values qss_jac_kernel computes (the same
// generated operations); the Jacobian's derivative terms are computed in
// FP32 and stored as FP64.  Own translation unit and cubin (the generated
// qss_eval_jac32, which uses qss_convert.h, is included before this file).
#pragma once

#include "qss_cells.cuh"

// Blocks per SM the register allocation must allow (1: up to 255 registers
// at 128 threads; 3: 168; 4: 128), a tuning option like QSS_MINBLOCKS of
// the FP64 kernel.
#ifndef QSS_J32_MINBLOCKS
#define QSS_J32_MINBLOCKS 1
#endif

extern "C" __global__ void __launch_bounds__(QSS_BLOCK, QSS_J32_MINBLOCKS)
qss_jac32_kernel(long long ncells, long long ld, const double* __restrict__ rho,
                 const double* __restrict__ T, const double* __restrict__ Y,
                 double* __restrict__ jac, double* __restrict__ wdot, double* __restrict__ Tdot,
                 const double* __restrict__ phi, const int* __restrict__ list,
                 const int* __restrict__ nact, int* __restrict__ nact_next) {
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double C[QSS_N];
  double Tc;
  double* jc;
  long long jstride;
  if (phi) {
    if (c == 0) *nact_next = 0;
    if (c >= *nact) return;
    QSS_DBG_CHECK(*nact <= ld, 1);
    const long long s = list[c];
    QSS_DBG_CHECK(s >= 0 && s < ld, 2);
#pragma unroll
    for (int k = 0; k < QSS_N; ++k) C[k] = phi[k * ld + s];
    Tc = phi[QSS_N * ld + s];
    jc = jac + (c >> 2) * (4 * QSS_JAC_NNZ) + (c & 3);
    jstride = 4;
  } else {
    if (c >= ncells) return;
    QSS_DBG_CHECK(c < ld, 3);
    qss_unpack(c, ld, rho, Y, C);
    Tc = __ldg(T + c);
    jc = jac + c;
    jstride = ld;
  }
  qss_eval_jac32(C, Tc, wdot ? wdot + c : nullptr, Tdot ? Tdot + c : nullptr, jc, ld, jstride);
}

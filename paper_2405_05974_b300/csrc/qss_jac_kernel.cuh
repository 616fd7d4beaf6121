// The analytic Jacobian kernel around a generated mechanism body (one thread
// per cell; the layout is in qss_cells.cuh).  It has a translation unit and a
// cubin of its own: the generated Jacobian is by far the longest compile, and
// it is redone only when this file or the mechanism changes.
#pragma once

#include "qss_cells.cuh"

// Blocks per SM the register allocation must allow for the Jacobian kernel
// (1: up to 255 registers; 2: <= 255 at 128 threads; 3: <= 168; 4: <= 128).
// Chosen per mechanism by the autotuner from timed variants.
#ifndef QSS_MINBLOCKS
#define QSS_MINBLOCKS 1
#endif

// f = (wdot, Tdot) and J.  State from (rho, T, Y) or, in list mode (phi and
// list given), of the t-th cell of the list: s = list[t] for t < *nact, state
// phi[k * ld + s] = (C_1..C_N, T), f written at column t (wdot[k * ld + t])
// and J written in groups of four cells, entry e of cell t at
// jac[(t / 4) * 4 * QSS_JAC_NNZ + 4 e + t % 4]: a warp's store of one entry
// fills eight whole 32-byte sectors, and the Newton update, whose warps take
// consecutive cells, reads each sector for four cells.  e is the entry's
// storage position: i (N+1) + j for a dense artefact, its index in the CSR
// value array for a CSR artefact (QSS_JAC_NNZ entries per cell either way).
// In list mode thread 0 also clears *nact_next, the counter the following
// Newton update fills.
extern "C" __global__ void __launch_bounds__(QSS_BLOCK, QSS_MINBLOCKS)
qss_jac_kernel(long long ncells, long long ld, const double* __restrict__ rho,
               const double* __restrict__ T, const double* __restrict__ Y,
               double* __restrict__ jac, double* __restrict__ wdot, double* __restrict__ Tdot,
               const double* __restrict__ phi, const int* __restrict__ list,
               const int* __restrict__ nact, int* __restrict__ nact_next) {
  QSS_SPILL_TO_SMEM();
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double C[QSS_N];
  double Tc;
  double* jc;
  long long jstride;
  if (phi) {
    if (c == 0) *nact_next = 0;
    if (c >= *nact) return;
    QSS_DBG_CHECK(*nact <= ld, 1);   // list positions index the ld-cell scratch
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
  // one call site: the generated body is inlined once
  qss_eval_jac(C, Tc, wdot ? wdot + c : nullptr, Tdot ? Tdot + c : nullptr, jc, ld, jstride);
}

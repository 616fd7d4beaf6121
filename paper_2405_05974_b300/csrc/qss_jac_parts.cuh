// The analytic Jacobian as a prefix kernel and column-group kernels (one
// thread per cell; the layout is in qss_cells.cuh).
//
// For a large mechanism the single generated Jacobian function is a very long
// straight-line program: its compile time grows faster than its length and
// its live values spill.  The mechanism compiler can instead split the DAG:
// the values needed by two or more column groups (rates, QSS
// concentrations, the production rates and their shared partial derivatives)
// are computed once per cell by the prefix kernel, which also writes wdot and
// Tdot, and stored to a frontier array; each column-group kernel reads the
// frontier values it needs and computes the rest of its Jacobian columns.
// Every DAG operation is computed exactly once.  Frontier layout, per cell c
// of a batch of `fld` cells: fr[slot * fld + c], slots 0..N-1 = C, N = T,
// then the prefix values.
//
// Each kernel has its own translation unit (QSS_JAC_PREFIX or QSS_JAC_GROUP
// defined, with the matching generated function) and its own cubin; the
// units compile in parallel.
#pragma once

#include "qss_cells.cuh"

#ifndef QSS_MINBLOCKS
#define QSS_MINBLOCKS 1
#endif

#ifdef QSS_JAC_PREFIX
// State from (rho, T, Y) or, in list mode (phi and list given), of the t-th
// cell of the list (s = list[t], t < *nact; state phi[k * ld + s]); wdot and
// Tdot written at column t with stride ld; thread 0 clears *nact_next in list
// mode (the counter the following Newton update fills).
extern "C" __global__ void __launch_bounds__(QSS_BLOCK)
qss_jac_prefix_kernel(long long ncells, long long ld, const double* __restrict__ rho,
                      const double* __restrict__ T, const double* __restrict__ Y,
                      double* __restrict__ wdot, double* __restrict__ Tdot, double* __restrict__ fr,
                      long long fld, const double* __restrict__ phi, const int* __restrict__ list,
                      const int* __restrict__ nact, int* __restrict__ nact_next) {
  QSS_SPILL_TO_SMEM();
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double C[QSS_N];
  double Tc;
  if (phi) {
    if (c == 0) *nact_next = 0;
    if (c >= *nact) return;
    QSS_DBG_CHECK(*nact <= ld && *nact <= fld, 1);
    const long long s = list[c];
    QSS_DBG_CHECK(s >= 0 && s < ld, 2);
#pragma unroll
    for (int k = 0; k < QSS_N; ++k) C[k] = phi[k * ld + s];
    Tc = phi[QSS_N * ld + s];
  } else {
    if (c >= ncells) return;
    QSS_DBG_CHECK(c < ld && c < fld, 3);
    qss_unpack(c, ld, rho, Y, C);
    Tc = __ldg(T + c);
  }
  qss_jac_prefix(C, Tc, wdot ? wdot + c : nullptr, Tdot ? Tdot + c : nullptr, ld, fr + c, fld);
}
#endif

#ifdef QSS_JAC_GROUP
// The group's Jacobian columns from the frontier of cell c.  With nact given
// (list mode) cells c < *nact are processed and J is written in groups of
// four cells, jac[(c / 4) * 4 * QSS_JAC_NNZ + 4 e + c % 4] (the Newton
// update's layout); otherwise cells c < ncells, jac[e * ld + c] (e: the
// entry's dense or CSR storage position).
extern "C" __global__ void __launch_bounds__(QSS_BLOCK, QSS_MINBLOCKS)
qss_jac_group_kernel(long long ncells, const double* __restrict__ fr, long long fld,
                     double* __restrict__ jac, long long ld, const int* __restrict__ nact) {
  QSS_SPILL_TO_SMEM();
  const long long c = (long long)blockIdx.x * QSS_BLOCK + threadIdx.x;
  double* jc;
  long long jstride;
  if (nact) {
    if (c >= *nact) return;
    QSS_DBG_CHECK(*nact <= fld && *nact <= ld, 1);
    jc = jac + (c >> 2) * (4 * QSS_JAC_NNZ) + (c & 3);
    jstride = 4;
  } else {
    if (c >= ncells) return;
    QSS_DBG_CHECK(c < fld && c < ld, 3);
    jc = jac + c;
    jstride = ld;
  }
  qss_jac_group(fr + c, fld, jc, jstride);
}
#endif

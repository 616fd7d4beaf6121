// The analytic Jacobian kernel with two cells per thread (build option
// cells_per_thread = 2; the layout is in qss_cells.cuh): each thread runs the
// generated two-cell body qss_eval_jac2, the one-cell body and its copy for a
// second cell interleaved, so that a warp has twice the independent work (and
// each thread twice the live values).  Same entry point, arguments, list mode
// and output layout as qss_jac_kernel.cuh; the runtime launches it over half
// the cells.
#pragma once

#include "qss_cells.cuh"

#ifndef QSS_MINBLOCKS
#define QSS_MINBLOCKS 1
#endif

extern "C" __global__ void __launch_bounds__(QSS_BLOCK, QSS_MINBLOCKS)
qss_jac_kernel(long long ncells, long long ld, const double* __restrict__ rho,
               const double* __restrict__ T, const double* __restrict__ Y,
               double* __restrict__ jac, double* __restrict__ wdot, double* __restrict__ Tdot,
               const double* __restrict__ phi, const int* __restrict__ list,
               const int* __restrict__ nact, int* __restrict__ nact_next) {
  QSS_SPILL_TO_SMEM();
  // block b takes cells 2 b BLOCK + tid and that + BLOCK, so that each warp
  // access of either cell is one contiguous segment; the grid covers
  // ncells / 2.  A second cell beyond the batch is evaluated as a copy of the
  // first with its outputs dropped (null pointers).
  const long long ca = (long long)blockIdx.x * (2 * QSS_BLOCK) + threadIdx.x;
  long long cb = ca + QSS_BLOCK;
  double Ca[QSS_N], Cb[QSS_N];
  double Ta, Tb;
  double *ja, *jb;
  long long jstride;
  bool hasb;
  if (phi) {
    if (ca == 0) *nact_next = 0;
    const long long na = *nact;
    if (ca >= na) return;
    QSS_DBG_CHECK(na <= ld, 1);
    hasb = cb < na;
    if (!hasb) cb = ca;
    const long long sa = list[ca], sb = list[cb];
    QSS_DBG_CHECK(sa >= 0 && sa < ld && sb >= 0 && sb < ld, 2);
#pragma unroll
    for (int k = 0; k < QSS_N; ++k) {
      Ca[k] = phi[k * ld + sa];
      Cb[k] = phi[k * ld + sb];
    }
    Ta = phi[QSS_N * ld + sa];
    Tb = phi[QSS_N * ld + sb];
    ja = jac + (ca >> 2) * (4 * QSS_JAC_NNZ) + (ca & 3);
    jb = jac + (cb >> 2) * (4 * QSS_JAC_NNZ) + (cb & 3);
    jstride = 4;
  } else {
    if (ca >= ncells) return;
    hasb = cb < ncells;
    if (!hasb) cb = ca;
    QSS_DBG_CHECK(ca < ld && cb < ld, 3);
    qss_unpack(ca, ld, rho, Y, Ca);
    qss_unpack(cb, ld, rho, Y, Cb);
    Ta = __ldg(T + ca);
    Tb = __ldg(T + cb);
    ja = jac + ca;
    jb = jac + cb;
    jstride = ld;
  }
  qss_eval_jac2(Ca, Ta, wdot ? wdot + ca : nullptr, Tdot ? Tdot + ca : nullptr, ja, Cb, Tb,
                (wdot && hasb) ? wdot + cb : nullptr, (Tdot && hasb) ? Tdot + cb : nullptr,
                hasb ? jb : nullptr, ld, jstride);
}

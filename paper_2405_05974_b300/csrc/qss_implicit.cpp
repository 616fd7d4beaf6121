// Implicit (backward-Euler) step: host side of qss_implicit_step.
//
// Per chunk of cells: setup, then max_iter x (Jacobian in phi mode, Newton
// update), then write-back; all enqueued on the caller's stream without
// synchronisation (converged cells return at once in later iterations).
#include <cuda.h>

#include <algorithm>

#include "qss_driver.h"
#include "qss_internal.h"

using namespace qss;

namespace {

}  // namespace

namespace qss {
struct NewtonOptsDev {   // layout of QssNewtonOpts in qss_newton.cuh
  int max_iter;
  double rtol, atol_C, atol_T;
  int max_refine;
  double refine_tol;
};
}  // namespace qss

namespace qss {
// The handle's Newton scratch for a call enqueued on `st`: at least `bytes`,
// reused only after the previous call's work (on any stream) is done with it
// -- st waits for the event the previous call recorded (the caller records it
// again with scratch_release once its work is enqueued).  One allocation
// attempt: QSS_ERR_OOM when the device cannot hold `bytes` (nothing is
// enqueued then, and the handle holds no scratch).
int scratch_acquire_bytes(qss_mech_s* m, size_t bytes, CUstream st) {
  if (m->newton_scratch_bytes < bytes) {
    if (m->newton_done) CU_TRY(drv().cuEventSynchronize(m->newton_done));
    if (m->newton_scratch) {
      drv().cuMemFree(m->newton_scratch);
      m->newton_scratch = 0;
      m->newton_scratch_bytes = 0;
    }
    if (drv().cuMemAlloc(&m->newton_scratch, bytes) != CUDA_SUCCESS) {
      m->newton_scratch = 0;
      return fail(QSS_ERR_OOM, "cannot allocate the Newton scratch");
    }
    m->newton_scratch_bytes = bytes;
  }
  if (!m->newton_done) CU_TRY(drv().cuEventCreate(&m->newton_done, CU_EVENT_DISABLE_TIMING));
  else CU_TRY(drv().cuStreamWaitEvent(st, m->newton_done, 0));
  return QSS_OK;
}

// The same for `*cells` cells of `per_cell` bytes (plus 256 bytes of
// alignment slack).  When the device cannot hold that much, the request is
// halved (whole waves, at least 32 cells) until an allocation succeeds;
// *cells is then the chunk the call runs in.
int scratch_acquire(qss_mech_s* m, size_t per_cell, int64_t* cells, CUstream st) {
  for (;;) {
    int rc = scratch_acquire_bytes(m, per_cell * (size_t)*cells + 256, st);
    if (rc != QSS_ERR_OOM) return rc;
    if (*cells <= 32) return fail(QSS_ERR_OOM, "cannot allocate the Newton scratch for 32 cells");
    *cells = chunk_cells(m, *cells / 2);
  }
}

int scratch_release(qss_mech_s* m, CUstream st) {
  CU_TRY(drv().cuEventRecord(m->newton_done, st));
  return QSS_OK;
}
}  // namespace qss

namespace qss {

size_t newton_scratch_per_cell(const qss_mech_s* m, int precision, bool reuse) {
  (void)precision;   // both forms keep J in FP64; the FP32 factors live in registers
  const int n = m->N + 1;
  const size_t base = (size_t)m->jac_nnz * sizeof(double) + (size_t)3 * n * sizeof(double) + 5 * sizeof(int) +
                      frontier_bytes_per_cell(m);
  // Jacobian reuse: the kept J, f of the cells that keep it, the previous
  // update norm, and the two lists of those cells
  return reuse ? base + (size_t)(m->jac_nnz + n + 1) * sizeof(double) + 2 * sizeof(int) : base;
}

int check_implicit_args(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                        const double* rho, double* T, double* Y, int precision,
                        const qss_newton_opts* opts, qss_newton_opts* o) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (ncells < 0 || ld < ncells) return fail(QSS_ERR_INVALID_ARG, "bad sizes (ncells < 0 or ld < ncells)");
  if (precision != QSS_LU_FP64 && precision != QSS_LU_FP32_IR && precision != QSS_LU_MIXED)
    return fail(QSS_ERR_INVALID_ARG, "unknown precision");
  if (dt_stride != 0 && dt_stride != 1) return fail(QSS_ERR_INVALID_ARG, "dt_stride must be 0 or 1");
  *o = {20, 1e-12, 1e-20, 1e-10, 10, 1e-8, 0};
  if (opts) *o = *opts;
  if (o->max_iter < 1 || o->max_refine < 0 || !(o->rtol >= 0) || !(o->atol_C >= 0) ||
      !(o->atol_T >= 0) || !(o->refine_tol >= 0) || (o->jac_reuse != 0 && o->jac_reuse != 1))
    return fail(QSS_ERR_INVALID_ARG, "bad Newton options");
  if (ncells == 0) return QSS_OK;
  if (!dt || !rho || !T || !Y) return fail(QSS_ERR_INVALID_ARG, "null array");
  if (!m->f_newton[lu_kind(precision)] || !m->f_newton_setup || !m->f_newton_finish)
    return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no Newton kernels");
  if (precision == QSS_LU_MIXED && !m->jac32)
    return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no mixed-precision Jacobian (jac32)");
  return QSS_OK;
}

// Enqueue one implicit step on `stream` using the given device scratch
// (scratch_bytes of it, 256-byte aligned), in chunks of as many cells as fit.
int implicit_launch(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                    const double* rho, double* T, double* Y, int precision,
                    const qss_newton_opts& o, int32_t* iters, int32_t* cell_status, CUstream st,
                    CUdeviceptr scratch, size_t scratch_bytes, const int* ncap, double* fn0,
                    double* fn1, const double* p0, int64_t p0ld) {
  if (ncells == 0) return QSS_OK;
  const int n = m->N + 1;
  // Jacobian reuse is for the implicit step's own solve (not the recorded
  // substeps of the integrator, which pass fn0 / fn1)
  const bool reuse = o.jac_reuse != 0 && !fn0 && !fn1;
  const size_t per_cell = newton_scratch_per_cell(m, precision, reuse);
  const int64_t cap = (int64_t)((scratch_bytes > 256 ? scratch_bytes - 256 : 0) / per_cell);
  if (cap < 32) return fail(QSS_ERR_BUDGET, "scratch too small for one warp of cells");
  int64_t chunk = std::min<int64_t>(cap / 32 * 32, (ncells + 31) / 32 * 32);
  if (chunk < ncells && !(ncap || fn0 || fn1 || p0)) chunk = chunk_cells(m, cap);   // whole waves per chunk
  if ((ncap || fn0 || fn1 || p0) && chunk < ncells)
    return fail(QSS_ERR_BUDGET, "a capped or recording launch must fit one chunk");
  NewtonOptsDev od = {o.max_iter, o.rtol, o.atol_C, o.atol_T, o.max_refine, o.refine_tol};
  const size_t S = (size_t)chunk;
  double* M64 = (double*)scratch;
  double* PHI = M64 + (size_t)m->jac_nnz * S;
  double* PHI0 = PHI + (size_t)n * S;
  double* F = PHI0 + (size_t)n * S;
  int* ACT = (int*)(F + (size_t)n * S);
  int* ST = ACT + S;
  int* IT = ST + S;
  int* LIST[2] = {IT + S, IT + 2 * S};
  int* NACT = IT + 3 * S;   // two counters (S is a multiple of 32, so they fit in the tail)
  // frontier of a partitioned Jacobian right after the two counters: ACT + 5 S
  // + 2 ints is 8-byte aligned (S % 32 == 0), and the region ends within
  // per_cell * S + 256 bytes of the scratch start
  double* FR = frontier_bytes_per_cell(m) ? (double*)(NACT + 2) : nullptr;
  // Jacobian reuse: after the frontier, the kept J of every cell (JK[s * nnz
  // + e]), f of the cells that keep theirs (F2, list positions), the
  // previous squared update norm (DN), their two lists and two counters
  double* JK = (double*)(NACT + 2) + frontier_bytes_per_cell(m) / sizeof(double) * S;
  double* F2 = JK + (size_t)m->jac_nnz * S;
  double* DN = F2 + (size_t)n * S;
  int* ULIST[2] = {(int*)(DN + S), (int*)(DN + S) + S};
  int* NU = ULIST[1] + S;
  long long sld = chunk, l = ld, pl = p0ld;
  int rc;
  int mode = 0;
  double* nulld = nullptr;
  int* nulli = nullptr;
  for (int64_t c0 = 0; c0 < ncells; c0 += chunk) {
    long long cells = std::min<int64_t>(chunk, ncells - c0), cc0 = c0;
    void* a_setup[] = {&cells, &cc0, &l, &rho, &T, &Y, &PHI, &PHI0, &ACT, &ST, &IT, &LIST[0], &NACT, &sld,
                       &ncap, &p0, &pl};
    if ((rc = launch_cells(m, m->f_newton_setup, cells, m->block, a_setup, st, 0))) return rc;
    if (reuse) CU_TRY(drv().cuMemsetD32Async((CUdeviceptr)NU, 0, 2, st));
    for (int it = 0; it < o.max_iter; ++it) {
      const int cur = it & 1, nxt = cur ^ 1;
      const int* lc = LIST[cur];
      const int* nc = NACT + cur;
      int* nn = NACT + nxt;
      if ((rc = jac_launch(m, cells, sld, nullptr, nullptr, nullptr, M64, F, F + (size_t)m->N * S, PHI,
                           lc, nc, nn, FR, (int64_t)S, st, precision == QSS_LU_MIXED)))
        return rc;
      int* l2 = LIST[nxt];
      if (!reuse) {
        void* a_upd[] = {&cc0, &dt, &dt_stride, &PHI, &PHI0, &F, &M64, &ACT, &ST, &IT,
                         &lc, &nc, &l2, &nn, &sld, &fn0, &fn1, &od, &mode, &nulld, &nulld, &nulli, &nulli};
        if ((rc = launch_update(m, precision, cells, a_upd, st))) return rc;
        continue;
      }
      // f alone for the cells that keep their Jacobian (list ULIST[cur])
      const int* ulc = ULIST[cur];
      const int* unc = NU + cur;
      int* unn = NU + nxt;
      int* ul2 = ULIST[nxt];
      const double* nullc = nullptr;
      double* F2T = F2 + (size_t)m->N * S;
      void* a_w[] = {&cells, &sld, &nullc, &nullc, &nullc, &F2, &F2T, &PHI, &ulc, &unc, &unn};
      if ((rc = launch_cells(m, m->f_wdot, cells, m->block, a_w, st, 0))) return rc;
      // fresh Jacobians (kept for the next iterations), then the kept ones
      int m1 = 1, m2 = 2;
      void* a_u1[] = {&cc0, &dt, &dt_stride, &PHI, &PHI0, &F, &M64, &ACT, &ST, &IT,
                      &lc, &nc, &l2, &nn, &sld, &fn0, &fn1, &od, &m1, &JK, &DN, &ul2, &unn};
      if ((rc = launch_update(m, precision, cells, a_u1, st))) return rc;
      void* a_u2[] = {&cc0, &dt, &dt_stride, &PHI, &PHI0, &F2, &M64, &ACT, &ST, &IT,
                      &ulc, &unc, &l2, &nn, &sld, &fn0, &fn1, &od, &m2, &JK, &DN, &ul2, &unn};
      if ((rc = launch_update(m, precision, cells, a_u2, st))) return rc;
    }
    void* a_fin[] = {&cells, &cc0, &l, &rho, &T, &Y, &PHI, &ST, &IT, &iters, &cell_status, &sld, &ncap};
    if ((rc = launch_cells(m, m->f_newton_finish, cells, m->block, a_fin, st, 0))) return rc;
  }
  return QSS_OK;
}

}  // namespace qss

extern "C" int qss_implicit_step(qss_mech_t m, int64_t ncells, int64_t ld, const double* dt,
                                 int dt_stride, const double* rho, double* T, double* Y,
                                 int precision, const qss_newton_opts* opts, int32_t* iters,
                                 int32_t* cell_status, void* stream) {
  qss_newton_opts o;
  int rc = check_implicit_args(m, ncells, ld, dt, dt_stride, rho, T, Y, precision, opts, &o);
  if (rc || ncells == 0) return rc;
  std::lock_guard<std::mutex> lock(m->mu);
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  const size_t per_cell = newton_scratch_per_cell(m, precision, o.jac_reuse != 0);
  int64_t cells = std::min<int64_t>(chunk_cells(m, (int64_t)(m->newton_budget / per_cell)),
                                    (ncells + 31) / 32 * 32);
  rc = scratch_acquire(m, per_cell, &cells, (CUstream)stream);
  if (rc) return rc;
  rc = implicit_launch(m, ncells, ld, dt, dt_stride, rho, T, Y, precision, o, iters, cell_status,
                       (CUstream)stream, m->newton_scratch, m->newton_scratch_bytes);
  int rr = scratch_release(m, (CUstream)stream);
  return rc ? rc : rr;
}

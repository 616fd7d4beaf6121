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
constexpr size_t kScratchBudget = size_t(4) << 30;   // bytes of Newton scratch per handle

struct NewtonOptsDev {   // layout of QssNewtonOpts in qss_newton.cuh
  int max_iter;
  double rtol, atol_C, atol_T;
  int max_refine;
  double refine_tol;
};

int ensure_scratch(qss_mech_s* m, size_t bytes) {
  if (m->newton_scratch_bytes >= bytes) return QSS_OK;
  if (m->newton_scratch) {
    drv().cuMemFree(m->newton_scratch);
    m->newton_scratch = 0;
    m->newton_scratch_bytes = 0;
  }
  CUresult r = drv().cuMemAlloc(&m->newton_scratch, bytes);
  if (r != CUDA_SUCCESS) return fail(QSS_ERR_OOM, "cannot allocate the Newton scratch");
  m->newton_scratch_bytes = bytes;
  return QSS_OK;
}
}  // namespace

extern "C" int qss_implicit_step(qss_mech_t m, int64_t ncells, int64_t ld, const double* dt,
                                 int dt_stride, const double* rho, double* T, double* Y,
                                 int precision, const qss_newton_opts* opts, int32_t* iters,
                                 int32_t* cell_status, void* stream) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (ncells < 0 || ld < ncells) return fail(QSS_ERR_INVALID_ARG, "bad sizes (ncells < 0 or ld < ncells)");
  if (precision != QSS_LU_FP64 && precision != QSS_LU_FP32_IR)
    return fail(QSS_ERR_INVALID_ARG, "unknown precision");
  if (dt_stride != 0 && dt_stride != 1) return fail(QSS_ERR_INVALID_ARG, "dt_stride must be 0 or 1");
  if (ncells == 0) return QSS_OK;
  if (!dt || !rho || !T || !Y) return fail(QSS_ERR_INVALID_ARG, "null array");
  if (!m->f_newton[precision] || !m->f_newton_setup || !m->f_newton_finish)
    return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no Newton kernels");
  qss_newton_opts o = {20, 1e-12, 1e-20, 1e-10, 10, 1e-14};
  if (opts) o = *opts;
  if (o.max_iter < 1 || o.max_refine < 0 || !(o.rtol >= 0) || !(o.atol_C >= 0) || !(o.atol_T >= 0) ||
      !(o.refine_tol >= 0))
    return fail(QSS_ERR_INVALID_ARG, "bad Newton options");
  NewtonOptsDev od = {o.max_iter, o.rtol, o.atol_C, o.atol_T, o.max_refine, o.refine_tol};
  std::lock_guard<std::mutex> lock(m->mu);
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  const int n = m->N + 1;
  const size_t per_cell = (size_t)n * n * (sizeof(double) + (precision ? sizeof(float) : 0)) +
                          (size_t)3 * n * sizeof(double) + 3 * sizeof(int);
  int64_t chunk = (int64_t)std::max<size_t>(kScratchBudget / per_cell, 32);
  chunk = std::min<int64_t>(chunk, (ncells + 31) / 32 * 32);
  chunk = (chunk + 31) / 32 * 32;
  int rc = ensure_scratch(m, per_cell * (size_t)chunk + 256);
  if (rc) return rc;
  const size_t S = (size_t)chunk;
  double* M64 = (double*)m->newton_scratch;
  double* PHI = M64 + (size_t)n * n * S;
  double* PHI0 = PHI + (size_t)n * S;
  double* F = PHI0 + (size_t)n * S;
  int* ACT = (int*)(F + (size_t)n * S);
  int* ST = ACT + S;
  int* IT = ST + S;
  float* M32 = precision ? (float*)(IT + S) : nullptr;
  long long sld = chunk, l = ld;
  CUstream st = (CUstream)stream;
  for (int64_t c0 = 0; c0 < ncells; c0 += chunk) {
    long long cells = std::min<int64_t>(chunk, ncells - c0), cc0 = c0;
    void* a_setup[] = {&cells, &cc0, &l, &rho, &T, &Y, &PHI, &PHI0, &ACT, &ST, &IT, &sld};
    if ((rc = launch_cells(m, m->f_newton_setup, cells, m->block, a_setup, st, 0))) return rc;
    const double* nul = nullptr;
    double* Fw = F;
    double* FT = F + (size_t)m->N * S;
    const double* phic = PHI;
    const int* actc = ACT;
    void* a_jac[] = {&cells, &sld, &nul, &nul, &nul, &M64, &Fw, &FT, &phic, &actc};
    void* a_upd[] = {&cells, &cc0, &dt, &dt_stride, &PHI, &PHI0, &F, &M64, &M32, &ACT, &ST, &IT, &sld, &od};
    for (int it = 0; it < o.max_iter; ++it) {
      if ((rc = launch_cells(m, m->f_jac, cells, m->block, a_jac, st, 0))) return rc;
      if ((rc = launch_cells(m, m->f_newton[precision], cells, m->block, a_upd, st, 0))) return rc;
    }
    void* a_fin[] = {&cells, &cc0, &l, &rho, &T, &Y, &PHI, &ST, &IT, &iters, &cell_status, &sld};
    if ((rc = launch_cells(m, m->f_newton_finish, cells, m->block, a_fin, st, 0))) return rc;
  }
  return QSS_OK;
}

// Implicit (backward-Euler) step: host side of qss_implicit_step.
#include <cuda.h>

#include "qss_internal.h"
#include "qss_driver.h"

using namespace qss;

extern "C" int qss_implicit_step(qss_mech_t m, int64_t ncells, int64_t ld, const double* dt,
                                 int dt_stride, const double* rho, double* T, double* Y,
                                 int precision, const qss_newton_opts* opts, int32_t* iters,
                                 int32_t* cell_status, void* stream) {
  (void)dt; (void)dt_stride; (void)rho; (void)T; (void)Y; (void)opts; (void)iters;
  (void)cell_status; (void)stream;
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (ncells < 0 || ld < ncells) return fail(QSS_ERR_INVALID_ARG, "bad sizes");
  if (precision != QSS_LU_FP64 && precision != QSS_LU_FP32_IR)
    return fail(QSS_ERR_INVALID_ARG, "unknown precision");
  if (!m->f_newton[precision]) return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no Newton kernel");
  return fail(QSS_ERR_UNIMPLEMENTED, "implicit step not built yet");
}

// qss_implicit_step_noalloc: the implicit step with its Newton scratch in a
// fixed device array instead of memory allocated by the library.
//
// Some callers cannot let a library allocate device memory: applications that
// reserve and manage all of the GPU's memory themselves (a flow solver sharing
// the device with its chemistry) and forbid hidden allocations, and loops that
// must not pay the device-wide synchronisation an allocation can imply.  This
// entry point allocates nothing: the Newton scratch is the file-scope array
// below, which every GPU that loads the library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "qss_driver.h"
#include "qss_internal.h"

using namespace qss;

// 64 MiB of Newton scratch (chunks of as many cells as fit: about 4000 cells
// of the 35+18-species workload per chunk).
#define QSS_NOALLOC_SCRATCH_BYTES (size_t(64) << 20)

static __device__ __align__(256) unsigned char qss_noalloc_scratch[QSS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
CUdeviceptr g_addr[kMaxDevices] = {};   // device address of the array, per device

// Once per device, with that device current: the array's device address.  In
// host code `qss_noalloc_scratch` names a host-side stand-in, not device
// memory, so it is never passed to a kernel directly.  The handle's context
// (the primary context of its device, which the CUDA runtime shares) is made
// current for the lookup, so no other device's context is created; a context
// that was current before is put back.
int scratch_address(qss_mech_s* m, CUdeviceptr* out) {
  if (m->device < 0 || m->device >= kMaxDevices) return fail(QSS_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[m->device]) {
    CUcontext prev = nullptr;
    if (drv().cuCtxGetCurrent(&prev) != CUDA_SUCCESS) prev = nullptr;
    CU_TRY(drv().cuCtxSetCurrent(m->ctx));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, qss_noalloc_scratch);
    if (prev && prev != m->ctx) drv().cuCtxSetCurrent(prev);
    if (e != cudaSuccess || !p)
      return fail(QSS_ERR_CUDA, std::string("cudaGetSymbolAddress(qss_noalloc_scratch): ") +
                                    cudaGetErrorString(e));
    g_addr[m->device] = (CUdeviceptr)p;
  }
  *out = g_addr[m->device];
  return QSS_OK;
}
}  // namespace

extern "C" int qss_implicit_step_noalloc(qss_mech_t m, int64_t ncells, int64_t ld, const double* dt,
                                         int dt_stride, const double* rho, double* T, double* Y,
                                         int precision, const qss_newton_opts* opts, int32_t* iters,
                                         int32_t* cell_status, void* stream) {
  qss_newton_opts o;
  int rc = check_implicit_args(m, ncells, ld, dt, dt_stride, rho, T, Y, precision, opts, &o);
  if (rc || ncells == 0) return rc;
  const size_t warp_chunk = newton_scratch_per_cell(m, precision, o.jac_reuse != 0) * 32 + 256;
  if (warp_chunk > QSS_NOALLOC_SCRATCH_BYTES)
    return fail(QSS_ERR_BUDGET, "mechanism too large for the fixed scratch: 32 cells need " +
                                    std::to_string(warp_chunk) + " bytes, the array holds " +
                                    std::to_string(QSS_NOALLOC_SCRATCH_BYTES));
  CUdeviceptr scratch = 0;
  if ((rc = scratch_address(m, &scratch))) return rc;
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  return implicit_launch(m, ncells, ld, dt, dt_stride, rho, T, Y, precision, o, iters, cell_status,
                         (CUstream)stream, scratch, QSS_NOALLOC_SCRATCH_BYTES);
}

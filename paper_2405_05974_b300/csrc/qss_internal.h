// Internal declarations shared by the runtime's translation units.
#pragma once
#include <cuda.h>

#include <mutex>
#include <string>
#include <vector>

#include "qss.h"

struct qss_mech_s {
  int device = 0;
  CUdevice dev = 0;
  CUcontext ctx = nullptr;
  CUmodule mod = nullptr;          // jac.cubin: analytic Jacobian kernel
  CUmodule mod_wdot = nullptr;     // wdot.cubin: source term, FD Jacobian
  CUmodule mod_newton = nullptr;   // newton.cubin: implicit-step kernels
  CUfunction f_wdot = nullptr, f_jac = nullptr, f_jac_fd = nullptr;
  CUfunction f_newton[2] = {nullptr, nullptr};   // update kernels: FP64 LU, FP32 LU + FP64 refinement
  CUfunction f_newton_setup = nullptr, f_newton_finish = nullptr;
  int upd_threads[2] = {128, 128};   // block size of the update kernels (their launch bound)
  int N = 0, Q = 0, M = 0, block = 0;
  std::vector<double> W;
  std::string name, digest, dir;
  // host-array path: two staging buffers and streams, one call at a time
  std::mutex mu;
  CUdeviceptr stage[2] = {0, 0};
  size_t stage_bytes = 0;
  CUstream st[2] = {nullptr, nullptr};
  // implicit step: Newton matrices of one chunk of cells (grown on demand)
  CUdeviceptr newton_scratch = 0;
  size_t newton_scratch_bytes = 0;
};

namespace qss {
extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
int cu_fail(CUresult r, const char* what);
std::string lib_dir();
int ctx_for_device(int device, CUdevice* dev, CUcontext* ctx);
int launch_cells(qss_mech_s* m, CUfunction f, int64_t ncells, int block, void** args,
                 CUstream stream, unsigned shmem);
// implicit step (qss_implicit.cpp)
size_t newton_scratch_per_cell(const qss_mech_s* m, int precision);
int check_implicit_args(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                        const double* rho, double* T, double* Y, int precision,
                        const qss_newton_opts* opts, qss_newton_opts* o);
int implicit_launch(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                    const double* rho, double* T, double* Y, int precision,
                    const qss_newton_opts& o, int32_t* iters, int32_t* cell_status, CUstream st,
                    CUdeviceptr scratch, size_t scratch_bytes);
}  // namespace qss

#define CU_TRY(call)                                   \
  do {                                                 \
    CUresult r__ = (call);                             \
    if (r__ != CUDA_SUCCESS) return qss::cu_fail(r__, #call); \
  } while (0)

// Internal declarations shared by the runtime's translation units.
#pragma once
#include <cuda.h>

#include <map>
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
  CUmodule mod_jac32 = nullptr;    // jac32.cubin: mixed-precision Jacobian (artefacts built with jac32)
  CUfunction f_wdot = nullptr, f_jac = nullptr, f_jac_fd = nullptr;   // f_wdot also has a list mode
  CUfunction f_jac32 = nullptr;    // qss_jac32_kernel (single-kernel artefacts built with jac32)
  int jac32 = 0;                   // meta.txt: the artefact carries the mixed-precision Jacobian
  int jac32_slots = 0;             // its FP32 values in dynamic shared memory (per thread)
  unsigned jac32_smem = 0;         // bytes of dynamic shared memory per block of qss_jac32_kernel
  CUfunction f_newton[2] = {nullptr, nullptr};   // update kernels: FP64 LU, FP32 LU + FP64 refinement
  CUfunction f_newton_setup = nullptr, f_newton_finish = nullptr;
  CUfunction f_integ[4] = {nullptr, nullptr, nullptr, nullptr};   // init, gather, accept, finish
  int upd_threads[2] = {128, 128};   // block size of the update kernels (their launch bound)
  int64_t upd_grid_max[2] = {0, 0};  // update blocks resident on the device at once (0: unknown)
  // partitioned Jacobian (jac_parts >= 2): prefix kernel + column-group kernels
  int jac_parts = 0, frontier = 0;   // frontier: doubles per cell between them
  CUmodule mod_prefix = nullptr;
  CUfunction f_prefix = nullptr;
  std::vector<CUmodule> mod_group;
  std::vector<CUfunction> f_group;
  // their mixed-precision forms (jac32_prefix.cubin, jac32_g<i>.cubin)
  CUmodule mod_prefix32 = nullptr;
  CUfunction f_prefix32 = nullptr;
  std::vector<CUmodule> mod_group32;
  std::vector<CUfunction> f_group32;
  // the column groups run side by side: group 0 on the caller's stream,
  // group i > 0 on gst[i - 1], forked after the prefix (ev_fork) and joined
  // back (ev_join) before anything later on the caller's stream; the fork
  // is enqueued under fork_mu (the streams and events are the handle's).
  // Empty gst: the groups run one after another on the caller's stream.
  std::vector<CUstream> gst;
  CUevent ev_fork = nullptr;
  std::vector<CUevent> ev_join;
  std::mutex fork_mu;
  // frontier scratch of the device-array path; fr_done orders its reuse
  // across streams (recorded after each call's last group kernel)
  CUdeviceptr fr_scratch = 0;
  int64_t fr_cells = 0;
  size_t fr_budget = size_t(4) << 30;   // bytes of that buffer (qss_mech_set_frontier_bytes;
                                        // set at load like newton_budget)
  CUevent fr_done = nullptr;
  int N = 0, Q = 0, M = 0, block = 0;
  // dynamic shared memory of the single Jacobian kernel (bytes per block):
  // smem_slots doubles per thread hold its most-reloaded values
  int smem_slots = 0;
  // cells per thread of the FP64 Jacobian kernel (1, or 2: its grid covers
  // half the cells)
  int cpt = 1;
  unsigned jac_smem = 0;
  // stored Jacobian entries per cell and their pattern (CSR; dense = all)
  int64_t jac_nnz = 0;
  std::vector<int32_t> jac_row_ptr, jac_col;
  int64_t wave_cells = 0;   // cells of one full wave of the Jacobian kernel (0: unknown)
  std::vector<double> W;
  std::string name, digest, dir;
  // cubin name -> path relative to the artefact directory (meta.txt "cubin"
  // lines: the artefacts of a mechanism share one copy of each cubin)
  std::map<std::string, std::string> cubin_path;
  // host-array path: two staging buffers and streams, one call at a time
  std::mutex mu;
  CUdeviceptr stage[2] = {0, 0};
  size_t stage_bytes = 0;
  CUstream st[2] = {nullptr, nullptr};
  // implicit step: Newton matrices of one chunk of cells (grown on demand)
  CUdeviceptr newton_scratch = 0;
  size_t newton_scratch_bytes = 0;
  CUevent newton_done = nullptr;   // recorded after each call's last use of the scratch
  // size limit of that scratch (qss_mech_set_newton_bytes; default 1/16 of
  // the device's memory, at most a quarter of the memory free at load):
  // larger chunks mean fewer Newton tails, the iterations in which only a
  // few slow cells are left
  size_t newton_budget = size_t(4) << 30;
};

namespace qss {
// The Newton update kernel of a precision (the mixed form factors like
// QSS_LU_FP32_IR; only its Jacobian kernel differs)
inline int lu_kind(int precision) { return precision == QSS_LU_MIXED ? QSS_LU_FP32_IR : precision; }
extern thread_local std::string g_err;
int fail(int code, const std::string& msg);
int cu_fail(CUresult r, const char* what);
std::string lib_dir();
int ctx_for_device(int device, CUdevice* dev, CUcontext* ctx);
int launch_cells(qss_mech_s* m, CUfunction f, int64_t ncells, int block, void** args,
                 CUstream stream, unsigned shmem);
// a Newton update kernel (precision 0 FP64, 1 FP32-IR, 2 mixed: the FP32-IR
// update) over a list of up to
// ncells cells: one warp per cell as far as the device holds such warps at
// once, the warps striding over the list beyond that
int launch_update(qss_mech_s* m, int precision, int64_t ncells, void** args, CUstream stream);
// wdot, Tdot and J of ncells cells, monolithic or partitioned.  State from
// (rho, T, Y) with leading dimension ld, J SoA with ld; or, in list mode (phi,
// list, nact given), of the listed cells with J cell-contiguous.  fr/fld: the
// frontier scratch of a partitioned Jacobian (fld >= ncells; unused
// otherwise).  mixed: the mixed-precision Jacobian kernel (the caller has
// checked that the artefact has it).
int jac_launch(qss_mech_s* m, int64_t ncells, int64_t ld, const double* rho, const double* T,
               const double* Y, double* jac, double* wdot, double* Tdot, const double* phi,
               const int* list, const int* nact, int* nact_next, double* fr, int64_t fld,
               CUstream s, bool mixed = false);
bool jac_pattern_ok(qss_mech_s* m);
// The chunk (in cells) for at most `cap` cells of scratch: a multiple of the
// Jacobian kernel's wave when at least one wave fits, else of 32 (>= 32).
int64_t chunk_cells(const qss_mech_s* m, int64_t cap);
inline size_t frontier_bytes_per_cell(const qss_mech_s* m) {
  return m->jac_parts >= 2 ? (size_t)m->frontier * sizeof(double) : 0;
}
// the handle's Newton scratch, ordered across streams (qss_implicit.cpp)
int scratch_acquire_bytes(qss_mech_s* m, size_t bytes, CUstream st);
int scratch_acquire(qss_mech_s* m, size_t per_cell, int64_t* cells, CUstream st);
int scratch_release(qss_mech_s* m, CUstream st);
// implicit step (qss_implicit.cpp)
// bytes of Newton scratch per cell; reuse: the Jacobian-reuse iteration's
// extra arrays (kept J, second f, previous norm, two more lists)
size_t newton_scratch_per_cell(const qss_mech_s* m, int precision, bool reuse = false);
int check_implicit_args(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                        const double* rho, double* T, double* Y, int precision,
                        const qss_newton_opts* opts, qss_newton_opts* o);
int implicit_launch(qss_mech_s* m, int64_t ncells, int64_t ld, const double* dt, int dt_stride,
                    const double* rho, double* T, double* Y, int precision,
                    const qss_newton_opts& o, int32_t* iters, int32_t* cell_status, CUstream st,
                    CUdeviceptr scratch, size_t scratch_bytes, const int* ncap = nullptr,
                    double* fn0 = nullptr, double* fn1 = nullptr, const double* p0 = nullptr,
                    int64_t p0ld = 0);
}  // namespace qss

#define CU_TRY(call)                                   \
  do {                                                 \
    CUresult r__ = (call);                             \
    if (r__ != CUDA_SUCCESS) return qss::cu_fail(r__, #call); \
  } while (0)

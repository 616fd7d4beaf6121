// libqss.so: host runtime of the B300 QSS chemistry library (C ABI in qss.h).
//
// Written against the CUDA driver API only: mechanism artefacts are cubins
// (sm_103a) loaded into the device's primary context, which the CUDA runtime
// (and PyTorch) share, so device pointers and streams pass through unchanged.
#include "qss.h"

#include <cuda.h>
#include <dlfcn.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <cmath>
#include <string>
#include <vector>

#include "qss_internal.h"
#include "qss_driver.h"

namespace qss {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cu_fail(CUresult r, const char* what) {
  const char* s = nullptr;
  if (drv().ok) drv().cuGetErrorString(r, &s);
  return fail(QSS_ERR_CUDA, std::string(what) + ": " + (s ? s : "unknown CUDA error"));
}

std::string lib_dir() {
  Dl_info info;
  if (dladdr((void*)&lib_dir, &info) && info.dli_fname) {
    std::string p(info.dli_fname);
    size_t k = p.rfind('/');
    return k == std::string::npos ? std::string(".") : p.substr(0, k);
  }
  return ".";
}

int ctx_for_device(int device, CUdevice* dev, CUcontext* ctx) {
  if (!drv().ok) return fail(QSS_ERR_CUDA, "CUDA driver (libcuda.so.1) is not available");
  CU_TRY(drv().cuInit(0));
  int count = 0;
  CU_TRY(drv().cuDeviceGetCount(&count));
  if (device < 0 || device >= count) return fail(QSS_ERR_INVALID_ARG, "device ordinal out of range");
  CU_TRY(drv().cuDeviceGet(dev, device));
  CU_TRY(drv().cuDevicePrimaryCtxRetain(ctx, *dev));
  CU_TRY(drv().cuCtxSetCurrent(*ctx));
  return QSS_OK;
}

int launch_cells(qss_mech_s* m, CUfunction f, int64_t ncells, int block, void** args,
                 CUstream stream, unsigned shmem) {
  if (ncells == 0) return QSS_OK;
  int64_t grid = (ncells + block - 1) / block;
  if (grid > INT_MAX) return fail(QSS_ERR_INVALID_ARG, "ncells too large for one launch");
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  CU_TRY(drv().cuLaunchKernel(f, (unsigned)grid, 1, 1, (unsigned)block, 1, 1, shmem, stream, args,
                        nullptr));
  return QSS_OK;
}

int launch_update(qss_mech_s* m, int precision, int64_t ncells, void** args, CUstream stream) {
  if (ncells == 0) return QSS_OK;
  precision = lu_kind(precision);
  const int block = m->upd_threads[precision], warps = std::max(block / 32, 1);
  // one warp per listed cell, capped at the blocks that are resident at once
  // (a small batch then spreads over every SM instead of queueing 32 cells
  // on each of ncells / 32 warps); without the occupancy figure, ncells / 32
  // warps as before
  int64_t grid = (ncells + warps - 1) / warps;
  if (m->upd_grid_max[precision] > 0) grid = std::min(grid, m->upd_grid_max[precision]);
  else grid = (ncells + block - 1) / block;
  if (grid > INT_MAX) return fail(QSS_ERR_INVALID_ARG, "ncells too large for one launch");
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  CU_TRY(drv().cuLaunchKernel(m->f_newton[precision], (unsigned)grid, 1, 1, (unsigned)block, 1, 1, 0, stream,
                              args, nullptr));
  return QSS_OK;
}

int64_t chunk_cells(const qss_mech_s* m, int64_t cap) {
  if (m->wave_cells > 0 && cap >= m->wave_cells) return cap / m->wave_cells * m->wave_cells;
  return std::max<int64_t>(32, cap / 32 * 32);
}

// Path of an artefact's cubin: the shared copy meta.txt names, else the file
// in the artefact directory.
static std::string cubin_file(const qss_mech_s* m, const std::string& dir, const std::string& name) {
  auto it = m->cubin_path.find(name);
  return dir + "/" + (it != m->cubin_path.end() ? it->second : name);
}

int jac_launch(qss_mech_s* m, int64_t ncells, int64_t ld, const double* rho, const double* T,
               const double* Y, double* jac, double* wdot, double* Tdot, const double* phi,
               const int* list, const int* nact, int* nact_next, double* fr, int64_t fld,
               CUstream s, bool mixed) {
  long long nc = ncells, l = ld;
  int rc;
  if (mixed && !m->jac32) return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no mixed-precision Jacobian (jac32)");
  if (mixed && m->jac_parts < 2) {
    void* args[] = {&nc, &l, &rho, &T, &Y, &jac, &wdot, &Tdot, &phi, &list, &nact, &nact_next};
    return launch_cells(m, m->f_jac32, ncells, m->block, args, s, m->jac32_smem);
  }
  if (m->jac_parts < 2) {
    void* args[] = {&nc, &l, &rho, &T, &Y, &jac, &wdot, &Tdot, &phi, &list, &nact, &nact_next};
    // with two cells per thread the grid covers half the cells
    return launch_cells(m, m->f_jac, (ncells + m->cpt - 1) / m->cpt, m->block, args, s, m->jac_smem);
  }
  if (!fr || fld < ncells) return fail(QSS_ERR_INVALID_ARG, "frontier scratch too small");
  long long fl = fld;
  void* pa[] = {&nc, &l, &rho, &T, &Y, &wdot, &Tdot, &fr, &fl, &phi, &list, &nact, &nact_next};
  const unsigned smem = mixed ? 0u : m->jac_smem;
  if ((rc = launch_cells(m, mixed ? m->f_prefix32 : m->f_prefix, ncells, m->block, pa, s, smem))) return rc;
  const double* frc = fr;
  // the groups only read the frontier and write disjoint Jacobian entries:
  // run them side by side (a few straggler cells in late Newton iterations
  // then cost one group's latency instead of K), joined back into s before
  // the frontier is written again
  const bool fork = (int)m->gst.size() == m->jac_parts - 1 && m->ev_fork;
  std::unique_lock<std::mutex> lk(m->fork_mu, std::defer_lock);
  if (fork) {
    lk.lock();
    CU_TRY(drv().cuEventRecord(m->ev_fork, s));
  }
  for (int i = 0; i < m->jac_parts; ++i) {
    void* ga[] = {&nc, &frc, &fl, &jac, &l, &nact};
    const CUstream gs = (fork && i > 0) ? m->gst[i - 1] : s;
    if (gs != s) CU_TRY(drv().cuStreamWaitEvent(gs, m->ev_fork, 0));
    if ((rc = launch_cells(m, mixed ? m->f_group32[i] : m->f_group[i], ncells, m->block, ga, gs, smem))) return rc;
    if (gs != s) CU_TRY(drv().cuEventRecord(m->ev_join[i - 1], gs));
  }
  if (fork)
    for (int i = 0; i + 1 < m->jac_parts; ++i) CU_TRY(drv().cuStreamWaitEvent(s, m->ev_join[i], 0));
  return QSS_OK;
}

// The stored Jacobian pattern from meta.txt: absent (older or dense
// artefacts) means dense, which is filled in here; a CSR pattern must have
// N + 2 row pointers from 0 to jac_nnz and strictly increasing columns in
// range within each row.
bool jac_pattern_ok(qss_mech_s* m) {
  const int n = m->N + 1;
  if (m->jac_row_ptr.empty() && m->jac_col.empty()) {
    if (m->jac_nnz != 0 && m->jac_nnz != (int64_t)n * n) return false;
    m->jac_nnz = (int64_t)n * n;
    for (int i = 0; i <= n; ++i) m->jac_row_ptr.push_back(i * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) m->jac_col.push_back(j);
    return true;
  }
  if ((int)m->jac_row_ptr.size() != n + 1 || m->jac_row_ptr[0] != 0 ||
      m->jac_row_ptr[n] != m->jac_nnz || (int64_t)m->jac_col.size() != m->jac_nnz ||
      m->jac_nnz <= 0 || m->jac_nnz > (int64_t)n * n)
    return false;
  for (int i = 0; i < n; ++i) {
    if (m->jac_row_ptr[i] > m->jac_row_ptr[i + 1]) return false;
    for (int p = m->jac_row_ptr[i]; p < m->jac_row_ptr[i + 1]; ++p)
      if (m->jac_col[p] < 0 || m->jac_col[p] >= n || (p > m->jac_row_ptr[i] && m->jac_col[p] <= m->jac_col[p - 1]))
        return false;
  }
  return true;
}

}  // namespace qss

using namespace qss;

extern "C" {

const char* qss_last_error(void) { return g_err.c_str(); }

int qss_mech_jac_pattern(qss_mech_t m, int64_t* nnz, const int32_t** row_ptr, const int32_t** col_idx) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (nnz) *nnz = m->jac_nnz;
  if (row_ptr) *row_ptr = m->jac_row_ptr.data();
  if (col_idx) *col_idx = m->jac_col.data();
  return QSS_OK;
}

int qss_mech_load(const char* artefact_dir, int device, qss_mech_t* out) {
  if (!artefact_dir || !out) return fail(QSS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  std::string dir(artefact_dir);
  std::ifstream meta(dir + "/meta.txt");
  if (!meta) return fail(QSS_ERR_MECH_FORMAT, "cannot open " + dir + "/meta.txt");
  qss_mech_s* m = new qss_mech_s();
  m->dir = dir;
  std::string line;
  while (std::getline(meta, line)) {
    std::istringstream ls(line);
    std::string key;
    ls >> key;
    if (key == "name") ls >> m->name;
    else if (key == "digest") ls >> m->digest;
    else if (key == "N") ls >> m->N;
    else if (key == "Q") ls >> m->Q;
    else if (key == "M") ls >> m->M;
    else if (key == "block") ls >> m->block;
    else if (key == "jac_parts") ls >> m->jac_parts;
    else if (key == "frontier") ls >> m->frontier;
    else if (key == "jac_nnz") ls >> m->jac_nnz;
    else if (key == "smem_slots") ls >> m->smem_slots;
    else if (key == "cpt") ls >> m->cpt;
    else if (key == "jac32") ls >> m->jac32;
    else if (key == "jac32_slots") ls >> m->jac32_slots;
    else if (key == "cubin") {
      std::string f, p;
      ls >> f >> p;
      m->cubin_path[f] = p;
    }
    else if (key == "jac_row_ptr" || key == "jac_col") {
      std::vector<int32_t>& v = key == "jac_col" ? m->jac_col : m->jac_row_ptr;
      int32_t x;
      while (ls >> x) v.push_back(x);
    } else if (key == "W") {
      double w;
      while (ls >> w) m->W.push_back(w);
    }
  }
  if (m->N <= 0 || m->Q < 0 || m->M <= 0 || m->block <= 0 || (int)m->W.size() != m->N ||
      m->jac_parts < 0 || m->jac_parts > 64 || (m->jac_parts >= 2 && m->frontier <= m->N) ||
      m->smem_slots < 0 || m->smem_slots > 1024 || m->cpt < 1 || m->cpt > 2 ||
      (m->cpt == 2 && (m->jac_parts >= 2 || m->smem_slots > 0)) ||
      m->jac32 < 0 || m->jac32 > 1 || m->jac32_slots < 0 || m->jac32_slots > 2048 ||
      (m->jac32_slots > 0 && (!m->jac32 || m->jac_parts >= 2)) ||
      !jac_pattern_ok(m)) {
    delete m;
    return fail(QSS_ERR_MECH_FORMAT, "inconsistent meta.txt in " + dir);
  }
  int rc = ctx_for_device(device, &m->dev, &m->ctx);
  if (rc) { delete m; return rc; }
  m->device = device;
  // required kernels: the analytic Jacobian (jac.cubin, or jac_prefix.cubin
  // and jac_g<i>.cubin when partitioned) and the source term with the
  // finite-difference Jacobian (wdot.cubin)
  struct Need { CUmodule* mod; std::string file; const char* fn; CUfunction* slot; };
  std::vector<Need> need;
  if (m->jac_parts >= 2) {
    m->mod_group.assign(m->jac_parts, nullptr);
    m->f_group.assign(m->jac_parts, nullptr);
    need.push_back({&m->mod_prefix, "jac_prefix.cubin", "qss_jac_prefix_kernel", &m->f_prefix});
    for (int i = 0; i < m->jac_parts; ++i)
      need.push_back({&m->mod_group[i], "jac_g" + std::to_string(i) + ".cubin", "qss_jac_group_kernel",
                      &m->f_group[i]});
    if (m->jac32) {
      m->mod_group32.assign(m->jac_parts, nullptr);
      m->f_group32.assign(m->jac_parts, nullptr);
      need.push_back({&m->mod_prefix32, "jac32_prefix.cubin", "qss_jac_prefix_kernel", &m->f_prefix32});
      for (int i = 0; i < m->jac_parts; ++i)
        need.push_back({&m->mod_group32[i], "jac32_g" + std::to_string(i) + ".cubin", "qss_jac_group_kernel",
                        &m->f_group32[i]});
    }
  } else {
    need.push_back({&m->mod, "jac.cubin", "qss_jac_kernel", &m->f_jac});
    if (m->jac32) need.push_back({&m->mod_jac32, "jac32.cubin", "qss_jac32_kernel", &m->f_jac32});
  }
  need.push_back({&m->mod_wdot, "wdot.cubin", "qss_wdot_kernel", &m->f_wdot});
  need.push_back({&m->mod_wdot, "wdot.cubin", "qss_jac_fd_kernel", &m->f_jac_fd});
  for (const Need& nd : need) {
    CUresult r = CUDA_SUCCESS;
    if (!*nd.mod) r = drv().cuModuleLoad(nd.mod, cubin_file(m, dir, nd.file).c_str());
    int code = 0;
    if (r != CUDA_SUCCESS) {
      code = cu_fail(r, ("drv().cuModuleLoad(" + nd.file + ")").c_str());
      *nd.mod = nullptr;
    } else if (drv().cuModuleGetFunction(nd.slot, *nd.mod, nd.fn) != CUDA_SUCCESS) {
      code = fail(QSS_ERR_MECH_FORMAT, std::string("artefact lacks kernel ") + nd.fn + " in " + nd.file);
    }
    if (code) {
      if (m->mod) drv().cuModuleUnload(m->mod);
      if (m->mod_jac32) drv().cuModuleUnload(m->mod_jac32);
      if (m->mod_wdot) drv().cuModuleUnload(m->mod_wdot);
      if (m->mod_prefix) drv().cuModuleUnload(m->mod_prefix);
      for (CUmodule g : m->mod_group)
        if (g) drv().cuModuleUnload(g);
      if (m->mod_prefix32) drv().cuModuleUnload(m->mod_prefix32);
      for (CUmodule g : m->mod_group32)
        if (g) drv().cuModuleUnload(g);
      drv().cuDevicePrimaryCtxRelease(m->dev);
      delete m;
      return code;
    }
  }
  if (m->smem_slots > 0) {
    // the FP64 Jacobian kernel (or the prefix and every column group of the
    // partitioned form) keeps smem_slots doubles per thread in shared memory
    m->jac_smem = (unsigned)m->smem_slots * (unsigned)m->block * sizeof(double);
    std::vector<CUfunction> fs = {m->jac_parts >= 2 ? m->f_prefix : m->f_jac};
    if (m->jac_parts >= 2) fs.insert(fs.end(), m->f_group.begin(), m->f_group.end());
    for (CUfunction f : fs) {
      CUresult ra = drv().cuFuncSetAttribute(f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                             (int)m->jac_smem);
      if (ra != CUDA_SUCCESS) {
        qss_mech_free(m);
        return cu_fail(ra, "cuFuncSetAttribute(Jacobian kernel, dynamic shared memory)");
      }
    }
  }
  if (m->jac32_slots > 0) {
    m->jac32_smem = (unsigned)m->jac32_slots * (unsigned)m->block * sizeof(float);
    CUresult ra = drv().cuFuncSetAttribute(m->f_jac32, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                                           (int)m->jac32_smem);
    if (ra != CUDA_SUCCESS) {
      qss_mech_free(m);
      return cu_fail(ra, "cuFuncSetAttribute(qss_jac32_kernel, dynamic shared memory)");
    }
  }
  // optional kernels (implicit step), in newton.cubin
  const char* opt[] = {"qss_newton_update_fp64_kernel", "qss_newton_update_fp32ir_kernel",
                       "qss_newton_setup_kernel", "qss_newton_finish_kernel"};
  CUfunction* oslot[] = {&m->f_newton[0], &m->f_newton[1], &m->f_newton_setup, &m->f_newton_finish};
  if (drv().cuModuleLoad(&m->mod_newton, cubin_file(m, dir, "newton.cubin").c_str()) != CUDA_SUCCESS)
    m->mod_newton = nullptr;
  for (int i = 0; i < 4; ++i)
    if (!m->mod_newton || drv().cuModuleGetFunction(oslot[i], m->mod_newton, opt[i]) != CUDA_SUCCESS)
      *oslot[i] = nullptr;
  const char* integ[] = {"qss_integ_init_kernel", "qss_integ_gather_kernel", "qss_integ_accept_kernel",
                         "qss_integ_finish_kernel"};
  for (int i = 0; i < 4; ++i)
    if (!m->mod_newton || drv().cuModuleGetFunction(&m->f_integ[i], m->mod_newton, integ[i]) != CUDA_SUCCESS)
      m->f_integ[i] = nullptr;
  for (int i = 0; i < 2; ++i) {
    int tpb = 0;
    if (m->f_newton[i] &&
        drv().cuFuncGetAttribute(&tpb, CU_FUNC_ATTRIBUTE_MAX_THREADS_PER_BLOCK, m->f_newton[i]) == CUDA_SUCCESS &&
        tpb > 0)
      m->upd_threads[i] = tpb;
  }
  // default scratch limits: 1/16 of the device's memory, but no more than a
  // quarter of what is free at load time (on a shared device, or when the
  // caller already holds most of the memory); allocation failures later halve
  // the chunk instead of failing the call
  size_t free_b = 0, total_b = 0;
  if (drv().cuMemGetInfo(&free_b, &total_b) == CUDA_SUCCESS && total_b > 0) {
    m->newton_budget = std::max<size_t>(size_t(64) << 20, std::min(total_b / 16, free_b / 4));
    m->fr_budget = m->newton_budget;
  }
  // cells of one full wave of the (first) Jacobian kernel: chunked paths use
  // multiples of it, so that no chunk ends in a partly filled wave
  int sms = 0, per_sm = 0;
  if (drv().cuDeviceGetAttribute(&sms, CU_DEVICE_ATTRIBUTE_MULTIPROCESSOR_COUNT, m->dev) != CUDA_SUCCESS)
    sms = 0;
  if (drv().cuOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, m->jac_parts >= 2 ? m->f_prefix : m->f_jac,
                                                        m->block, m->jac_smem) != CUDA_SUCCESS)
    per_sm = 0;
  m->wave_cells = (int64_t)std::max(sms, 0) * std::max(per_sm, 0) * m->block * (m->jac_parts >= 2 ? 1 : m->cpt);
  for (int i = 0; i < 2; ++i) {
    int upd_per_sm = 0;
    if (m->f_newton[i] && sms > 0 &&
        drv().cuOccupancyMaxActiveBlocksPerMultiprocessor(&upd_per_sm, m->f_newton[i], m->upd_threads[i], 0) ==
            CUDA_SUCCESS)
      m->upd_grid_max[i] = (int64_t)sms * std::max(upd_per_sm, 0);
  }
  // streams and events of the side-by-side column groups (without them the
  // groups run in sequence)
  if (m->jac_parts >= 2) {
    bool ok = drv().cuEventCreate(&m->ev_fork, CU_EVENT_DISABLE_TIMING) == CUDA_SUCCESS;
    for (int i = 0; ok && i + 1 < m->jac_parts; ++i) {
      CUstream st = nullptr;
      CUevent ev = nullptr;
      ok = drv().cuStreamCreate(&st, CU_STREAM_NON_BLOCKING) == CUDA_SUCCESS;
      if (ok) m->gst.push_back(st);
      ok = ok && drv().cuEventCreate(&ev, CU_EVENT_DISABLE_TIMING) == CUDA_SUCCESS;
      if (ok) m->ev_join.push_back(ev);
    }
    if (!ok) {   // partial set: release it and run the groups in sequence
      for (CUstream st : m->gst) drv().cuStreamDestroy(st);
      for (CUevent ev : m->ev_join) drv().cuEventDestroy(ev);
      if (m->ev_fork) drv().cuEventDestroy(m->ev_fork);
      m->gst.clear();
      m->ev_join.clear();
      m->ev_fork = nullptr;
    }
  }
  *out = m;
  return QSS_OK;
}

void qss_mech_free(qss_mech_t m) {
  if (!m) return;
  drv().cuCtxSetCurrent(m->ctx);
  for (int b = 0; b < 2; ++b) {
    if (m->stage[b]) drv().cuMemFree(m->stage[b]);
    if (m->st[b]) drv().cuStreamDestroy(m->st[b]);
  }
  if (m->newton_scratch) drv().cuMemFree(m->newton_scratch);
  if (m->newton_done) drv().cuEventDestroy(m->newton_done);
  if (m->fr_scratch) drv().cuMemFree(m->fr_scratch);
  if (m->fr_done) drv().cuEventDestroy(m->fr_done);
  for (CUstream st : m->gst) drv().cuStreamDestroy(st);
  for (CUevent ev : m->ev_join) drv().cuEventDestroy(ev);
  if (m->ev_fork) drv().cuEventDestroy(m->ev_fork);
  if (m->mod_prefix) drv().cuModuleUnload(m->mod_prefix);
  for (CUmodule g : m->mod_group)
    if (g) drv().cuModuleUnload(g);
  if (m->mod_prefix32) drv().cuModuleUnload(m->mod_prefix32);
  for (CUmodule g : m->mod_group32)
    if (g) drv().cuModuleUnload(g);
  if (m->mod) drv().cuModuleUnload(m->mod);
  if (m->mod_jac32) drv().cuModuleUnload(m->mod_jac32);
  if (m->mod_wdot) drv().cuModuleUnload(m->mod_wdot);
  if (m->mod_newton) drv().cuModuleUnload(m->mod_newton);
  drv().cuDevicePrimaryCtxRelease(m->dev);
  delete m;
}

int qss_mech_info(qss_mech_t m, int* n_transported, int* n_qss, int* n_reactions,
                  const double** W_host) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (n_transported) *n_transported = m->N;
  if (n_qss) *n_qss = m->Q;
  if (n_reactions) *n_reactions = m->M;
  if (W_host) *W_host = m->W.data();
  return QSS_OK;
}

static int check_cells(qss_mech_t m, int64_t ncells, int64_t ld) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (ncells < 0) return fail(QSS_ERR_INVALID_ARG, "ncells < 0");
  if (ld < ncells) return fail(QSS_ERR_INVALID_ARG, "ld < ncells");
  return QSS_OK;
}

int qss_wdot(qss_mech_t m, int64_t ncells, int64_t ld, const double* rho, const double* T,
             const double* Y, double* wdot, double* Tdot, void* stream) {
  int rc = check_cells(m, ncells, ld);
  if (rc) return rc;
  if (ncells == 0) return QSS_OK;
  if (!rho || !T || !Y || !wdot) return fail(QSS_ERR_INVALID_ARG, "null array");
  long long nc = ncells, l = ld;
  const double* phi = nullptr;
  const int *list = nullptr, *nact = nullptr;
  int* nact_next = nullptr;
  void* args[] = {&nc, &l, &rho, &T, &Y, &wdot, &Tdot, &phi, &list, &nact, &nact_next};
  return launch_cells(m, m->f_wdot, ncells, m->block, args, (CUstream)stream, 0);
}

static int jacobian_impl(qss_mech_t m, int64_t ncells, int64_t ld, const double* rho, const double* T,
                         const double* Y, double* jac, double* wdot, double* Tdot, void* stream, bool mixed) {
  int rc = check_cells(m, ncells, ld);
  if (rc) return rc;
  if (mixed && !m->jac32) return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no mixed-precision Jacobian (jac32)");
  if (ncells == 0) return QSS_OK;
  if (!rho || !T || !Y || !jac) return fail(QSS_ERR_INVALID_ARG, "null array");
  CUstream s = (CUstream)stream;
  if (m->jac_parts < 2)
    return jac_launch(m, ncells, ld, rho, T, Y, jac, wdot, Tdot, nullptr, nullptr, nullptr, nullptr,
                      nullptr, 0, s, mixed);
  // partitioned: chunks of cells through the handle's frontier scratch (at
  // most fr_budget bytes), its reuse ordered after the previous call by an
  // event
  std::lock_guard<std::mutex> lock(m->mu);
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  const size_t per = frontier_bytes_per_cell(m);
  int64_t want = std::min<int64_t>(chunk_cells(m, (int64_t)(m->fr_budget / per)), (ncells + 31) / 32 * 32);
  if (m->fr_cells > want && (int64_t)(m->fr_budget / per) < m->fr_cells) {
    // the budget was lowered: give the larger buffer back
    if (m->fr_done) CU_TRY(drv().cuEventSynchronize(m->fr_done));
    drv().cuMemFree(m->fr_scratch);
    m->fr_scratch = 0;
    m->fr_cells = 0;
  }
  if (m->fr_cells < want) {
    if (m->fr_done) CU_TRY(drv().cuEventSynchronize(m->fr_done));
    if (m->fr_scratch) { drv().cuMemFree(m->fr_scratch); m->fr_scratch = 0; m->fr_cells = 0; }
    // the device may hold less than the limit: halve the chunk (down to 32
    // cells) until the buffer fits, and lower the limit to what fitted (so
    // that qss_jacobian_launches stays exact and later calls do not retry)
    bool halved = false;
    while (drv().cuMemAlloc(&m->fr_scratch, per * (size_t)want) != CUDA_SUCCESS) {
      m->fr_scratch = 0;
      if (want <= 32) return fail(QSS_ERR_OOM, "cannot allocate the Jacobian frontier scratch for 32 cells");
      want = chunk_cells(m, want / 2);
      halved = true;
    }
    if (halved) m->fr_budget = per * (size_t)want;
    m->fr_cells = want;
  }
  want = std::min(want, m->fr_cells);
  if (!m->fr_done) CU_TRY(drv().cuEventCreate(&m->fr_done, CU_EVENT_DISABLE_TIMING));
  else CU_TRY(drv().cuStreamWaitEvent(s, m->fr_done, 0));
  double* fr = (double*)m->fr_scratch;
  for (int64_t c0 = 0; c0 < ncells; c0 += want) {
    const int64_t cs = std::min<int64_t>(want, ncells - c0);
    if ((rc = jac_launch(m, cs, ld, rho + c0, T + c0, Y + c0, jac + c0, wdot ? wdot + c0 : nullptr,
                         Tdot ? Tdot + c0 : nullptr, nullptr, nullptr, nullptr, nullptr, fr,
                         m->fr_cells, s, mixed)))
      return rc;
  }
  CU_TRY(drv().cuEventRecord(m->fr_done, s));
  return QSS_OK;
}

int qss_jacobian(qss_mech_t m, int64_t ncells, int64_t ld, const double* rho, const double* T,
                 const double* Y, double* jac, double* wdot, double* Tdot, void* stream) {
  return jacobian_impl(m, ncells, ld, rho, T, Y, jac, wdot, Tdot, stream, false);
}

int qss_jacobian_mixed(qss_mech_t m, int64_t ncells, int64_t ld, const double* rho, const double* T,
                       const double* Y, double* jac, double* wdot, double* Tdot, void* stream) {
  return jacobian_impl(m, ncells, ld, rho, T, Y, jac, wdot, Tdot, stream, true);
}

int qss_debug_status(qss_mech_t m, int* status) {
  if (!m || !status) return fail(QSS_ERR_INVALID_ARG, "null argument");
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  std::vector<CUmodule> mods = {m->mod, m->mod_wdot, m->mod_newton, m->mod_prefix};
  mods.insert(mods.end(), m->mod_group.begin(), m->mod_group.end());
  bool any = false;
  int first = 0;
  for (CUmodule mod : mods) {
    CUdeviceptr p = 0;
    size_t bytes = 0;
    if (!mod || drv().cuModuleGetGlobal(&p, &bytes, mod, "qss_debug_word") != CUDA_SUCCESS) continue;
    any = true;
    int v = 0;
    CU_TRY(drv().cuMemcpyDtoHAsync(&v, p, sizeof(int), nullptr));
    CU_TRY(drv().cuStreamSynchronize(nullptr));
    if (v && !first) first = v;
    if (v) {
      CU_TRY(drv().cuMemsetD32Async(p, 0, 1, nullptr));
      CU_TRY(drv().cuStreamSynchronize(nullptr));
    }
  }
  if (!any) return fail(QSS_ERR_UNIMPLEMENTED, "the artefact is not a QSS_DEBUG build");
  *status = first;
  return QSS_OK;
}

int qss_mech_set_newton_bytes(qss_mech_t m, size_t bytes) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  std::lock_guard<std::mutex> lock(m->mu);
  m->newton_budget = bytes;
  return QSS_OK;
}

int qss_jacobian_launches(qss_mech_t m, int64_t ncells, int64_t* launches) {
  if (!m || !launches || ncells < 0) return fail(QSS_ERR_INVALID_ARG, "bad argument");
  if (ncells == 0) { *launches = 0; return QSS_OK; }
  if (m->jac_parts < 2) { *launches = 1; return QSS_OK; }
  const size_t per = frontier_bytes_per_cell(m);
  const int64_t want = std::min<int64_t>(chunk_cells(m, (int64_t)(m->fr_budget / per)), (ncells + 31) / 32 * 32);
  *launches = (ncells + want - 1) / want * (m->jac_parts + 1);
  return QSS_OK;
}

int qss_mech_set_frontier_bytes(qss_mech_t m, size_t bytes) {
  if (!m) return fail(QSS_ERR_INVALID_ARG, "null mechanism");
  if (m->jac_parts >= 2 && bytes < 32 * frontier_bytes_per_cell(m))
    return fail(QSS_ERR_INVALID_ARG, "frontier buffer smaller than 32 cells");
  std::lock_guard<std::mutex> lock(m->mu);
  m->fr_budget = bytes;
  return QSS_OK;
}

int qss_jacobian_fd(qss_mech_t m, int64_t ncells, int64_t ld, const double* rho,
                    const double* T, const double* Y, double dC, double dT, double* jac,
                    void* stream) {
  int rc = check_cells(m, ncells, ld);
  if (rc) return rc;
  if (!(dC > 0.0) || !(dT > 0.0) || !std::isfinite(dC) || !std::isfinite(dT))
    return fail(QSS_ERR_INVALID_ARG, "finite-difference steps must be finite and > 0");
  if (ncells == 0) return QSS_OK;
  if (!rho || !T || !Y || !jac) return fail(QSS_ERR_INVALID_ARG, "null array");
  long long nc = ncells, l = ld;
  void* args[] = {&nc, &l, &rho, &T, &Y, &dC, &dT, &jac};
  return launch_cells(m, m->f_jac_fd, ncells, m->block, args, (CUstream)stream, 0);
}

static int copy2d(void* dst, bool dst_host, size_t dpitch, const void* src, bool src_host,
                  size_t spitch, size_t width, size_t height, CUstream s) {
  CUDA_MEMCPY2D c;
  std::memset(&c, 0, sizeof(c));
  if (src_host) {
    c.srcMemoryType = CU_MEMORYTYPE_HOST;
    c.srcHost = src;
  } else {
    c.srcMemoryType = CU_MEMORYTYPE_DEVICE;
    c.srcDevice = (CUdeviceptr)src;
  }
  if (dst_host) {
    c.dstMemoryType = CU_MEMORYTYPE_HOST;
    c.dstHost = dst;
  } else {
    c.dstMemoryType = CU_MEMORYTYPE_DEVICE;
    c.dstDevice = (CUdeviceptr)dst;
  }
  c.srcPitch = spitch;
  c.dstPitch = dpitch;
  c.WidthInBytes = width;
  c.Height = height;
  CU_TRY(drv().cuMemcpy2DAsync(&c, s));
  return QSS_OK;
}

int qss_jacobian_host(qss_mech_t m, int64_t ncells, const double* rho, const double* T,
                      const double* Y, double* jac, double* wdot, double* Tdot, int64_t chunk,
                      void* stream) {
  (void)stream;
  int rc = check_cells(m, ncells, ncells);
  if (rc) return rc;
  if (ncells == 0) return QSS_OK;
  if (!rho || !T || !Y || !jac) return fail(QSS_ERR_INVALID_ARG, "null array");
  std::lock_guard<std::mutex> lock(m->mu);
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  const int N = m->N;
  int64_t S = chunk > 0 ? chunk : 65536;
  S = std::min<int64_t>(S, ncells);
  S = (S + 31) / 32 * 32;
  const size_t fpc = frontier_bytes_per_cell(m) / sizeof(double);
  const size_t nnz = (size_t)m->jac_nnz;
  const size_t per_cell = (size_t)(2 + N + N + 1) + nnz + fpc;
  const size_t need = per_cell * (size_t)S * sizeof(double);
  if (m->stage_bytes < need) {
    for (int b = 0; b < 2; ++b) {
      if (m->stage[b]) { drv().cuMemFree(m->stage[b]); m->stage[b] = 0; }
      CUresult r = drv().cuMemAlloc(&m->stage[b], need);
      if (r != CUDA_SUCCESS) {
        m->stage_bytes = 0;
        return fail(QSS_ERR_OOM, "cannot allocate host-path staging buffers");
      }
    }
    m->stage_bytes = need;
  }
  for (int b = 0; b < 2; ++b)
    if (!m->st[b]) CU_TRY(drv().cuStreamCreate(&m->st[b], CU_STREAM_NON_BLOCKING));
  const size_t P = (size_t)S * sizeof(double);
  int64_t nchunks = (ncells + S - 1) / S;
  for (int64_t ci = 0; ci < nchunks; ++ci) {
    int b = (int)(ci & 1);
    CUstream s = m->st[b];
    int64_t c0 = ci * S;
    int64_t cs = std::min<int64_t>(S, ncells - c0);
    double* base = (double*)m->stage[b];
    double* d_rho = base;
    double* d_T = base + S;
    double* d_Y = base + 2 * S;
    double* d_w = base + (2 + N) * S;
    double* d_Td = base + (2 + 2 * N) * S;
    double* d_J = base + (3 + 2 * N) * S;
    const size_t w = (size_t)cs * sizeof(double), hp = (size_t)ncells * sizeof(double);
    if ((rc = copy2d(d_rho, false, P, rho + c0, true, hp, w, 1, s))) return rc;
    if ((rc = copy2d(d_T, false, P, T + c0, true, hp, w, 1, s))) return rc;
    if ((rc = copy2d(d_Y, false, P, Y + c0, true, hp, w, N, s))) return rc;
    double* d_fr = d_J + nnz * S;   // frontier (partitioned Jacobian only)
    if ((rc = jac_launch(m, cs, S, d_rho, d_T, d_Y, d_J, d_w, d_Td, nullptr, nullptr, nullptr,
                         nullptr, fpc ? d_fr : nullptr, S, s)))
      return rc;
    if ((rc = copy2d(jac + c0, true, hp, d_J, false, P, w, nnz, s))) return rc;
    if (wdot && (rc = copy2d(wdot + c0, true, hp, d_w, false, P, w, N, s))) return rc;
    if (Tdot && (rc = copy2d(Tdot + c0, true, hp, d_Td, false, P, w, 1, s))) return rc;
  }
  CU_TRY(drv().cuStreamSynchronize(m->st[0]));
  CU_TRY(drv().cuStreamSynchronize(m->st[1]));
  return QSS_OK;
}

}  // extern "C"

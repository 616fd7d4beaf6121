// Integration over an interval by backward-Euler or variable-step BDF2
// substeps with local error control: host side of qss_integrate.
//
// Per chunk of cells: an init kernel, then rounds of (gather the active cells
// into a contiguous batch, with the constant term of a BDF2 substep; one
// Newton-solved substep of the batch with each cell's own step h, recording f at the step's start and at
// the last Newton iterate; accept or reject each substep and build the next
// active list), then a kernel that writes the step counts and statuses.  The
// active counts stay on the device (the Newton kernels read them), so the
// rounds are enqueued without synchronisation; every 8 rounds the host reads
// the count and stops once no cell is left.
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "qss_driver.h"
#include "qss_internal.h"

using namespace qss;

namespace {

constexpr int kCheckEvery = 8;                     // rounds between host checks of the count

struct IntegOptsDev {   // layout of QssIntegOpts in qss_newton.cuh
  double rtol, atol_C, atol_T;
  double h_min;
  int order;
};

// per-cell bytes: persistent (TT, HH, DT, HP; PP, FP [n] each; IS, NS, LA,
// LB), batch (rho, T, dt, Y[N]; status; FN0, FN1, PC [n] each) and the Newton
// scratch of the batch
size_t integ_per_cell(const qss_mech_s* m, int prec) {
  const int N = m->N, n = N + 1;
  return (size_t)(4 + 2 * n + 3 + N + 3 * n) * sizeof(double) + 5 * sizeof(int) +
         newton_scratch_per_cell(m, prec);
}

}  // namespace

extern "C" int qss_integrate(qss_mech_t m, int64_t ncells, int64_t ld, const double* dt_total,
                             int dt_stride, const double* rho, double* T, double* Y, int precision,
                             const qss_integrate_opts* opts, int32_t* nsteps, int32_t* cell_status,
                             void* stream) {
  // substep Newton: at most 6 iterations (a substep that needs more is retried
  // smaller, which costs less than iterating on: every iteration is a full
  // Jacobian evaluation, and stiff cells that fail fail at any cap)
  qss_integrate_opts io = {1e-4, 1e-10, 1e-4, 0.0, 1e-14, 400, {6, 1e-12, 1e-20, 1e-10, 10, 1e-8, 0}, 1};
  if (opts) io = *opts;
  qss_newton_opts o;
  int rc = check_implicit_args(m, ncells, ld, dt_total, dt_stride, rho, T, Y, precision, &io.newton, &o);
  if (rc || ncells == 0) return rc;
  if (!(io.rtol >= 0) || !(io.atol_C > 0) || !(io.atol_T > 0) || !(io.h0 >= 0) ||
      !(io.h_min > 0 && io.h_min < 1e-12) || io.max_rounds < 1 || (io.order != 1 && io.order != 2))
    return fail(QSS_ERR_INVALID_ARG,
                "bad integration options (atol > 0, 0 < h_min < 1e-12, order 1 or 2 required)");
  for (int k = 0; k < 4; ++k)
    if (!m->f_integ[k]) return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no integration kernels");
  std::lock_guard<std::mutex> lock(m->mu);
  CU_TRY(drv().cuCtxSetCurrent(m->ctx));
  CUstream st = (CUstream)stream;
  const int N = m->N, n = N + 1;
  const size_t per = integ_per_cell(m, precision);
  int64_t S = std::min<int64_t>(chunk_cells(m, (int64_t)(m->newton_budget / per)), (ncells + 31) / 32 * 32);
  // layout (offsets in bytes, every array 256-byte aligned) for a chunk of S
  // cells; S is halved (whole waves, at least 32 cells) while the device
  // cannot hold the scratch
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t D, I, off;
  auto take = [&](size_t b) { size_t o0 = off; off += b; return o0; };
  size_t oTT, oHH, oDT, oIS, oNS, oLA, oLB, oCNT, oRb, oTb, oDtb, oYb, oBst, oF0, oF1, oHP, oPP, oFP, oPC,
      oNewton;
  for (;;) {
    D = al((size_t)S * sizeof(double));
    I = al((size_t)S * sizeof(int));
    off = 0;
    oTT = take(D); oHH = take(D); oDT = take(D); oIS = take(I); oNS = take(I);
    oLA = take(I); oLB = take(I); oCNT = take(256);
    oRb = take(D); oTb = take(D); oDtb = take(D); oYb = take((size_t)N * D);
    oBst = take(I); oF0 = take((size_t)n * D); oF1 = take((size_t)n * D);
    oHP = take(D); oPP = take((size_t)n * D); oFP = take((size_t)n * D); oPC = take((size_t)n * D);
    oNewton = take(0);
    const size_t total = off + newton_scratch_per_cell(m, precision) * (size_t)S + 256;
    rc = scratch_acquire_bytes(m, total, st);
    if (rc != QSS_ERR_OOM) break;
    if (S <= 32) return fail(QSS_ERR_OOM, "cannot allocate the integration scratch for 32 cells");
    S = chunk_cells(m, S / 2);
  }
  if (rc) return rc;
  const size_t newton_bytes = newton_scratch_per_cell(m, precision) * (size_t)S + 256;
  char* base = (char*)m->newton_scratch;
  double* TT = (double*)(base + oTT);
  double* HH = (double*)(base + oHH);
  double* DTv = (double*)(base + oDT);
  int* IS = (int*)(base + oIS);
  int* NS = (int*)(base + oNS);
  int* L[2] = {(int*)(base + oLA), (int*)(base + oLB)};
  int* CNT = (int*)(base + oCNT);   // [0], [1]: list counts; [2]: the batch's cell count
  double* rhob = (double*)(base + oRb);
  double* Tb = (double*)(base + oTb);
  double* dtb = (double*)(base + oDtb);
  double* Yb = (double*)(base + oYb);
  int* bst = (int*)(base + oBst);
  double* F0 = (double*)(base + oF0);
  double* F1 = (double*)(base + oF1);
  double* HP = (double*)(base + oHP);   // order 2: previous substep, phi_n-1, f_n-1, constant term
  double* PP = (double*)(base + oPP);
  double* FP = (double*)(base + oFP);
  double* PC = (double*)(base + oPC);
  const double* P0 = io.order == 2 ? PC : nullptr;
  CUdeviceptr newton = m->newton_scratch + oNewton;
  IntegOptsDev od = {io.rtol, io.atol_C, io.atol_T, io.h_min, io.order};
  long long bld = S, l = ld, SS = S;
  int order = io.order;
  for (int64_t c0 = 0; c0 < ncells; c0 += S) {
    long long cells = std::min<int64_t>(S, ncells - c0), cc0 = c0;
    double h0 = io.h0;
    int* CA = CNT;
    int* ncap = CNT + 2;
    void* a_init[] = {&cells, &cc0, &dt_total, &dt_stride, &h0, &TT, &HH, &DTv, &IS, &NS, &L[0], &CA, &HP};
    if ((rc = launch_cells(m, m->f_integ[0], cells, m->block, a_init, st, 0))) break;
    for (int round = 0; round < io.max_rounds; ++round) {
      const int a = round & 1, b = a ^ 1;
      int* LA = L[a];
      int* LB = L[b];
      int* ca = CNT + a;
      int* cb = CNT + b;
      void* a_g[] = {&cc0, &l, &rho, &T, &Y, &LA, &ca, &cb, &HH, &rhob, &Tb, &Yb, &dtb, &ncap, &bld,
                     &HP, &PP, &PC, &SS, &order};
      if ((rc = launch_cells(m, m->f_integ[1], cells, m->block, a_g, st, 0))) break;
      if ((rc = implicit_launch(m, cells, bld, dtb, 1, rhob, Tb, Yb, precision, o, nullptr, bst, st,
                                newton, newton_bytes, ncap, F0, F1, P0, bld)))
        break;
      void* a_a[] = {&cc0, &l, &T, &Y, &LA, &ca, &LB, &cb, &HH, &TT, &DTv, &IS, &NS,
                     &rhob, &Tb, &Yb, &bst, &F0, &F1, &bld, &od, &HP, &PP, &FP, &SS};
      if ((rc = launch_cells(m, m->f_integ[2], cells, m->block, a_a, st, 0))) break;
      if ((round + 1) % kCheckEvery == 0) {
        int left = 0;
        CUresult r1 = drv().cuMemcpyDtoHAsync(&left, (CUdeviceptr)cb, sizeof(int), st);
        if (r1 == CUDA_SUCCESS) r1 = drv().cuStreamSynchronize(st);
        if (r1 != CUDA_SUCCESS) { rc = cu_fail(r1, "integration count read-back"); break; }
        if (left == 0) break;
      }
    }
    if (rc) break;
    void* a_f[] = {&cells, &cc0, &IS, &NS, &nsteps, &cell_status};
    if ((rc = launch_cells(m, m->f_integ[3], cells, m->block, a_f, st, 0))) break;
  }
  int rr = scratch_release(m, st);
  return rc ? rc : rr;
}

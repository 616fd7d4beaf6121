/*
 * qss.h -- C ABI of the B300 QSS chemistry library (libqss.so).
 *
 * The library evaluates, per computational cell, the net production rates
 * (wdot) of a quasi-steady-state (QSS) reduced reaction mechanism and the
 * analytic chemical Jacobian of f = (wdot, Tdot) with respect to
 * phi = (C_1..C_N, T), and advances cells by one implicit backward-Euler step.
 * References are to Hassanaly et al., "Symbolic construction of the chemical
 * Jacobian of quasi-steady state (QSS) chemistries for Exascale computing
 * platforms":
 *   rates of progress / production rates ... Section 2.1, Eqs. (progRates), (ReacMech)
 *   QSS relations and their linear system .. Section 2.1 Eq. (QSSi), Section 2.3 Eq. (full_QSSsystem)
 *   resolution order (Tarjan SCC) .......... Section 2.3, Appendix B
 *   state vector and Jacobian .............. Section 3.1, Eq. (JacExptr)
 *   chain rule through C_QSS ............... Section 3.2, Eq. (JQSS)
 *   symbolic construction with CSE ......... Section 3.2.2
 *   simplified Jacobians, FD Jacobian ...... Section 3.2.1, Eq. (frobErr); FD T column 3.2.2
 *   implicit steps and integration ......... Section 3.1 (the stiff 0D use the Jacobian serves)
 * The mechanism compiler (paper_2405_05974_b300.qssc) produces the artefacts
 * this library loads; linearization of quadratic QSS couplings (Section 2.2,
 * Alg. 1) and the Jacobian variants are compiler options.
 *
 * Conventions shared by every entry point
 *   - Units are SI: rho kg/m^3, T K, concentrations mol/m^3, wdot mol/m^3/s,
 *     Tdot K/s, time s.
 *   - Arrays are FP64 structure-of-arrays with a leading dimension ld >= ncells:
 *       rho[c], T[c], Tdot[c]            c < ncells
 *       Y[k * ld + c], wdot[k * ld + c]  k < N (transported species only)
 *       jac[(i * (N+1) + j) * ld + c]    row i = d f_i, column j = d/d phi_j,
 *                                        index N stands for temperature
 *                                        (dense artefacts; a CSR artefact
 *                                        stores jac[p * ld + c] for the
 *                                        entries of qss_mech_jac_pattern).
 *   - "Device" arrays are device pointers on the mechanism's device; "host"
 *     arrays are host pointers (page-locked memory gives full copy speed).
 *   - The caller owns every array; the library never frees or retains one
 *     beyond the call.  Only a mechanism's module and its staging buffers, and
 *     a server's queues and buffers, belong to the library.
 *   - Device-array calls are asynchronous on `stream` (a CUstream /
 *     cudaStream_t of the mechanism's device; NULL = the legacy default
 *     stream) and return once the work is enqueued.
 *   - Return values report argument, launch and allocation errors (qss_status);
 *     qss_last_error() gives a message for the calling thread.  Per-cell
 *     numerical failures of the implicit step are reported in cell_status and
 *     never abort the launch.
 *   - ncells == 0 is valid and does nothing.
 */
#ifndef QSS_H
#define QSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qss_mech_s* qss_mech_t;
typedef struct qss_server_s* qss_server_t;

typedef enum {
  QSS_OK = 0,
  QSS_ERR_INVALID_ARG = -1,   /* null pointer, ld < ncells, unknown option      */
  QSS_ERR_MECH_FORMAT = -2,   /* unreadable or inconsistent artefact             */
  QSS_ERR_CUDA = -3,          /* a CUDA driver call failed (message has details) */
  QSS_ERR_OOM = -4,           /* device or host allocation failed                */
  QSS_ERR_NOT_CONVERGED = -5, /* reserved                                        */
  QSS_ERR_TIMEOUT = -6,       /* a wait exceeded its time limit                  */
  QSS_ERR_BUDGET = -7,        /* request larger than the server's memory budget  */
  QSS_ERR_UNIMPLEMENTED = -8
} qss_status;

/* Precision of the implicit step's Newton systems: FP64 LU; FP32 LU with
 * FP64 residual refinement; the same FP32-IR solve of a matrix whose
 * Jacobian's derivative terms were assembled in FP32 (qss_jacobian_mixed). */
enum { QSS_LU_FP64 = 0, QSS_LU_FP32_IR = 1, QSS_LU_MIXED = 2 };

/* Per-cell outcome of qss_implicit_step. */
enum {
  QSS_CELL_CONVERGED = 0,   /* Newton converged                              */
  QSS_CELL_MAXITER = 1,     /* iteration cap reached                         */
  QSS_CELL_NONFINITE = 2,   /* an iterate or residual became NaN/Inf         */
  QSS_CELL_SINGULAR = 3     /* zero pivot in the Newton matrix                */
};

/* ---------------------------------------------------------------------------
 * Mechanisms.  An artefact directory is produced by the mechanism compiler
 * (paper_2405_05974_b300.qssc): jac.cubin, wdot.cubin, newton.cubin (sm_103a)
 * and meta.txt.
 * qss_mech_load loads it on `device` (the primary context, shared with the
 * CUDA runtime) and returns a handle owned by the caller, released with
 * qss_mech_free.  Errors: QSS_ERR_INVALID_ARG (null arguments),
 * QSS_ERR_MECH_FORMAT (missing/inconsistent files), QSS_ERR_CUDA.
 * ------------------------------------------------------------------------- */
int qss_mech_load(const char* artefact_dir, int device, qss_mech_t* out);
void qss_mech_free(qss_mech_t mech);

/* Sizes of a loaded mechanism and its molar masses W[N] (kg/mol; the pointer
 * stays valid until qss_mech_free).  Any output pointer may be NULL. */
int qss_mech_info(qss_mech_t mech, int* n_transported, int* n_qss, int* n_reactions,
                  const double** W_host);

/* The stored Jacobian entries of a mechanism: nnz per cell, and their
 * pattern in CSR form (row_ptr[N+2], col_idx[nnz], columns increasing within a
 * row; the arrays stay valid until qss_mech_free).  A dense artefact stores
 * every entry (nnz = (N+1)^2, position i (N+1) + j); an artefact built with
 * the CSR format stores only the structural nonzeros of the generated
 * Jacobian (entries whose expression is not identically zero: the nonzero
 * pattern of Table memQSS, Sec. 3.2.3), entry p of row i at column
 * col_idx[p], row_ptr[i] <= p < row_ptr[i+1].  qss_jacobian and
 * qss_jacobian_host then write nnz rows of ld (or ncells) values instead of
 * (N+1)^2; qss_jacobian_fd stays dense.  Any output pointer may be NULL. */
int qss_mech_jac_pattern(qss_mech_t mech, int64_t* nnz, const int32_t** row_ptr,
                         const int32_t** col_idx);

/* Production rates (Eqs. progRates, ReacMech, with the QSS concentrations from
 * Eq. full_QSSsystem solved in SCC order).  Device arrays rho, T, Y (inputs),
 * wdot [N][ld] (output), Tdot [ld] (output, may be NULL). */
int qss_wdot(qss_mech_t mech, int64_t ncells, int64_t ld, const double* rho, const double* T,
             const double* Y, double* wdot, double* Tdot, void* stream);

/* Analytic Jacobian, Eq. (JacExptr) with the chain rule of Eq. (JQSS), of
 * f = (wdot, Tdot) with respect to phi = (C, T), constant volume.  Device
 * arrays; jac [nnz][ld] is required (nnz = (N+1)^2 for a dense artefact, see
 * qss_mech_jac_pattern), wdot [N][ld] and Tdot [ld] may be NULL (they are
 * computed anyway). */
/* Mixed-precision form of qss_jacobian for the Newton iteration matrix
 * (same arguments, layouts and outputs).  Everything the source term needs --
 * Arrhenius exponentials, equilibrium constants, third bodies and falloff,
 * the QSS solve of Eq. full_QSSsystem, the rates of progress -- is evaluated
 * in FP64 by the operations of qss_jacobian, so wdot and Tdot are its FP64
 * values (to within the reassociation the compiler may apply); the nodes only
 * the Jacobian needs (the rate derivatives, dC_Q/dphi and the chain-rule
 * products of Eq. JQSS) are evaluated in FP32 and stored as doubles.  Each
 * entry's error is bounded to first order by 2^29 times the FP64 rounding
 * bound of the same evaluation (the unit-roundoff ratio), about 1e-7 of the
 * entry where its terms do not cancel.  The paper evaluates the Jacobian in
 * FP64 throughout; this form serves implicit solvers, where J only shapes the
 * Newton matrix and the FP64 residual fixes the solution.  Errors: as
 * qss_jacobian; QSS_ERR_UNIMPLEMENTED if the artefact was built without the
 * mixed-precision kernel (build option jac32). */
int qss_jacobian_mixed(qss_mech_t mech, int64_t ncells, int64_t ld, const double* rho,
                       const double* T, const double* Y, double* jac, double* wdot, double* Tdot,
                       void* stream);

int qss_jacobian(qss_mech_t mech, int64_t ncells, int64_t ld, const double* rho,
                 const double* T, const double* Y, double* jac, double* wdot, double* Tdot,
                 void* stream);

/* Which Jacobian qss_jacobian computes is fixed when the artefact is built:
 * the exact one above (default), or the simplified ones of Section 3.2.1
 * (constant-QSS: the second term of Eq. JQSS dropped; zero-QSS: that term
 * dropped and the QSS concentrations set to zero inside the Jacobian), each
 * with the temperature column analytic or by the central difference of
 * Section 3.2.2 (step h = 2^(e-20) for T in [2^e, 2^(e+1))).  The row of T
 * follows from the species rows by the chain rule in every variant. */

/* A mechanism built with a partitioned Jacobian (a prefix kernel and column-
 * group kernels exchanging per-cell values through a frontier buffer) runs
 * qss_jacobian in chunks of cells that fit that buffer, which the handle owns
 * and keeps.  This sets its size limit in bytes (default 1/16 of the device's
 * memory, but at most a quarter of the memory free when the mechanism was
 * loaded, at least 64 MiB; larger chunks mean fewer launches).  When the
 * device cannot hold the buffer, qss_jacobian halves the chunk (down to 32
 * cells) and lowers the limit to what fitted.  No effect for a single-kernel
 * Jacobian.  Errors: QSS_ERR_INVALID_ARG if the limit holds fewer than 32
 * cells.
 * The column groups of each chunk run side by side: the first on the
 * caller's stream, the others on streams the handle creates at load, forked
 * by an event recorded on the caller's stream after the prefix kernel and
 * joined back into it before the call returns, so the call stays ordered on
 * the caller's stream (and a stream capture records the groups as parallel
 * branches).  The fork is enqueued under a lock of the handle. */
int qss_mech_set_frontier_bytes(qss_mech_t mech, size_t bytes);

/* Size limit in bytes of the handle's Newton scratch, used by
 * qss_implicit_step and qss_integrate (batches larger than the limit run in
 * chunks, each with its own tail of Newton iterations in which few cells are
 * left).  Default: 1/16 of the device's memory, but at most a quarter of the
 * memory free when the mechanism was loaded, at least 64 MiB.  A chunk holds
 * at least 32 cells whatever the limit; the scratch is allocated on first use
 * and kept (freed by qss_mech_free); when the device cannot hold it, the
 * chunk is halved (down to 32 cells) before QSS_ERR_OOM is returned. */
int qss_mech_set_newton_bytes(qss_mech_t mech, size_t bytes);

/* Bounds-check status of a QSS_DEBUG artefact (built with the preprocessor
 * definition QSS_DEBUG=1; a debugging aid, the paper has no counterpart).  In
 * such a build every kernel checks each index it forms into the caller's
 * arrays and the library's scratch against the extents it was given, before
 * the access; a violation skips the access and records a nonzero code in a
 * device status word instead of trapping, so the context stays usable.
 * Codes: 1 active-list count beyond the scratch, 2 list entry out of range,
 * 3 cell beyond ld (or the frontier's extent), 4 chunk larger than the
 * Newton scratch, 5 cell beyond the state arrays, 6 Newton active count out
 * of range, 7 Newton list entry out of range.  *status receives the first
 * code recorded since the last call (0: none) and the word is cleared.  Call
 * it after the checked work has completed (the read is ordered on the legacy
 * default stream only).  Errors: QSS_ERR_UNIMPLEMENTED for a release
 * artefact. */
int qss_debug_status(qss_mech_t mech, int* status);

/* Number of kernel launches qss_jacobian makes for ncells cells with the
 * handle's current frontier limit: 1 for a single-kernel Jacobian, (chunks) x
 * (groups + 1) for a partitioned one (for launch accounting).  Errors:
 * QSS_ERR_INVALID_ARG for a null handle or output, or ncells < 0. */
int qss_jacobian_launches(qss_mech_t mech, int64_t ncells, int64_t* launches);

/* Central finite-difference Jacobian of f = (wdot, Tdot), the reference of
 * Eq. (frobErr): column j = (f(phi + h e_j) - f(phi - h e_j)) / (2h), with the
 * absolute step h = dC (mol/m^3) for the concentration columns and h = dT (K)
 * for the temperature column.  Dense layout [(N+1)^2][ld] whatever the
 * artefact's storage format, otherwise the same arrays as qss_jacobian; costs
 * 2(N+1) source-term evaluations per cell.  Errors: QSS_ERR_INVALID_ARG for
 * null arrays or steps that are not finite and positive. */
int qss_jacobian_fd(qss_mech_t mech, int64_t ncells, int64_t ld, const double* rho,
                    const double* T, const double* Y, double dC, double dT, double* jac,
                    void* stream);

/* The same as qss_jacobian for HOST arrays with ld = ncells.  The batch is
 * processed in chunks of `chunk` cells (0 = automatic) through two device
 * staging buffers owned by the mechanism handle, with host->device copies,
 * kernels and device->host copies of consecutive chunks overlapped on two
 * streams.  Synchronous: returns when all outputs are in host memory.
 * `stream` is unused (reserved).  Errors: QSS_ERR_OOM if the staging buffers
 * cannot be allocated. */
int qss_jacobian_host(qss_mech_t mech, int64_t ncells, const double* rho, const double* T,
                      const double* Y, double* jac, double* wdot, double* Tdot, int64_t chunk,
                      void* stream);

/* ---------------------------------------------------------------------------
 * Implicit step.  One backward-Euler step at constant volume (rho fixed) of
 * dC/dt = wdot, dT/dt = Tdot: Newton on G(phi) = phi - phi0 - dt f(phi) with
 * the matrix I - dt J (the analytic Jacobian re-evaluated every iteration).
 * The Newton update is accepted when its weighted RMS norm with weights
 * 1 / (rtol |phi_i| + atol_i) is <= 1.  precision = QSS_LU_FP64 factors the
 * matrix with partial pivoting in FP64; QSS_LU_FP32_IR factors it in FP32
 * and refines the solution with FP64 residuals until the correction is below
 * refine_tol relative (or max_refine sweeps); a cell whose FP32
 * factorisation meets a zero or non-finite pivot, or whose refinement turns
 * non-finite, is solved in FP64 for that iteration instead, so the mixed form
 * reports QSS_CELL_SINGULAR only where the FP64 form would.  QSS_LU_MIXED
 * solves as QSS_LU_FP32_IR with J from qss_jacobian_mixed (derivative terms
 * in FP32): an inexact Newton iteration whose FP64 residual G fixes the root,
 * so a converged cell meets the same stopping rule; it may take an iteration
 * more.  Rates, equilibrium constants, the QSS solve and the Newton residual
 * stay FP64 in every form.
 * T [ld] and Y [N][ld] are updated in place (device arrays); dt is a device
 * array [ld] (dt_stride = 1) or a single device value (dt_stride = 0).
 * iters and cell_status (device int32 [ld]) may be NULL.
 * ------------------------------------------------------------------------- */
typedef struct {
  int max_iter;        /* Newton iteration cap (default 20)                 */
  double rtol;         /* default 1e-12                                      */
  double atol_C;       /* mol/m^3, default 1e-20                             */
  double atol_T;       /* K, default 1e-10                                   */
  int max_refine;      /* FP32_IR refinement sweeps (default 10)             */
  double refine_tol;   /* FP32_IR relative correction target (default 1e-8)  */
  int jac_reuse;       /* 0 (default): full Newton, the analytic Jacobian    */
                       /* every iteration; 1: keep a cell's Jacobian while   */
                       /* its Newton update norm shrinks by 0.3x or more per */
                       /* iteration (only f is evaluated then, and the       */
                       /* iteration matrix is refactored from the kept J);   */
                       /* a slower contraction evaluates a fresh Jacobian.   */
                       /* A kept-J update whose norm grows is discarded and  */
                       /* the cell retries with a fresh Jacobian.  The       */
                       /* converged state satisfies the same stopping rule;  */
                       /* these iterations converge linearly, so allow more  */
                       /* of them (max_iter about 40).                       */
} qss_newton_opts;

int qss_implicit_step(qss_mech_t mech, int64_t ncells, int64_t ld, const double* dt,
                      int dt_stride, const double* rho, double* T, double* Y, int precision,
                      const qss_newton_opts* opts, int32_t* iters, int32_t* cell_status,
                      void* stream);

/* ---------------------------------------------------------------------------
 * Integration over an interval.  Advances every cell by dt_total (device
 * array with dt_stride 1, or a scalar with dt_stride 0) at constant volume
 * with substeps under local error control, the kind of stiff integration
 * over a CFD substep the paper's Jacobian serves (Section 3.1, which drives
 * CVODE; this is not CVODE).  Each substep of size h is solved by Newton
 * (qss_implicit_step's solver) from phi_n:
 *   order 1: backward Euler, phi - phi_n - h f(phi) = 0, local error
 *            e = h/2 (f(phi_n+1) - f(phi_n));
 *   order 2: variable-step BDF2 once a substep has been accepted (the first
 *            is backward Euler): with w = h / h_prev,
 *            phi - a1 phi_n - a2 phi_n-1 - beta h f(phi) = 0, a1 =
 *            (1+w)^2/(1+2w), a2 = -w^2/(1+2w), beta = (1+w)/(1+2w); local
 *            error e = h (1+w)/(3(1+2w)) ((f(phi_n+1) - f(phi_n)) - w (f(phi_n)
 *            - f(phi_n-1))), its truncation error with the third derivative
 *            from divided differences of f,
 * with f at the last Newton iterate standing for f(phi_n+1).  A substep is
 * accepted when the weighted RMS err of e with weights rtol |phi_i| + atol_i
 * is <= 1; the next h is h min(g_max, max(0.2, 0.9 err^(-1/(p+1)))) for a
 * substep of order p (g_max 4 for order 1, 2 for order 2, inside BDF2's
 * step-ratio stability bound; capped by what remains of the interval).  A
 * rejected substep retries with h max(0.2, min(0.9, 0.9 err^(-1/(p+1)))), a
 * failed Newton solve with h / 4.  T and Y (device arrays) are
 * updated in place; nsteps [ld] receives the accepted substeps and
 * cell_status [ld] 0 (interval done), 1 (max_rounds substep attempts
 * exhausted; T, Y hold the last accepted state) or 2 (h fell below h_min x
 * dt_total).  Synchronises with the host every 8 rounds (to stop once every
 * cell is done).  Errors: as qss_implicit_step, QSS_ERR_INVALID_ARG for bad
 * options.
 * ------------------------------------------------------------------------- */
typedef struct {
  double rtol, atol_C, atol_T;   /* substep error tolerance (defaults 1e-4, 1e-10, 1e-4) */
  double h0;                     /* first substep in s (0: 1 % of the interval)     */
  double h_min;                  /* smallest substep / interval (default 1e-14)     */
  int max_rounds;                /* substep attempts per cell (default 400)         */
  qss_newton_opts newton;        /* each substep's Newton solve (default max_iter 6; */
                                 /* jac_reuse is not used by the substeps)          */
  int order;                     /* 1 backward Euler (default), 2 variable-step BDF2 */
} qss_integrate_opts;

int qss_integrate(qss_mech_t mech, int64_t ncells, int64_t ld, const double* dt_total,
                  int dt_stride, const double* rho, double* T, double* Y, int precision,
                  const qss_integrate_opts* opts /* nullable */, int32_t* nsteps,
                  int32_t* cell_status, void* stream);

/* ---------------------------------------------------------------------------
 * Serving (continuous batching of implicit-step requests on one GPU).
 *
 * qss_serve_create allocates a device arena of budget_bytes (the memory
 * budget) and starts a scheduler thread with n_streams streams.  A request is
 * one backward-Euler step (qss_implicit_step semantics, dt a scalar) of
 * `ncells` cells given in HOST arrays with leading dimension ncells: rho
 * [ncells], T [ncells] and Y [N][ncells] (updated in place when the request
 * completes), iters / cell_status [ncells] (may be NULL).  The arrays must stay
 * valid and untouched until qss_serve_wait returns for the request (page-locked
 * memory gives full copy speed).  Queued requests are admitted in arrival
 * order as soon as a stream slot and arena memory are free; queued requests of
 * the same mechanism and precision are merged into one launch of up to
 * max_batch_cells cells.  Per-cell results do not depend on the batch a request
 * lands in.  Errors at submit: QSS_ERR_BUDGET if the request alone exceeds the
 * budget or max_batch_cells.  qss_serve_wait blocks until the request is done
 * (timeout_us < 0: no limit; otherwise QSS_ERR_TIMEOUT after timeout_us and the
 * request stays pending); it returns the request's status and releases its id.
 * qss_serve_destroy finishes queued and running work, then frees everything.
 * ------------------------------------------------------------------------- */
typedef struct {
  int n_streams;                   /* concurrent batches (default 4)              */
  int64_t max_batch_cells;         /* cells per merged launch (default 262144)    */
  const qss_newton_opts* newton;   /* NULL: qss_implicit_step defaults            */
  int graphs;                      /* 0: default = on; 1: on; -1: off (see below) */
} qss_serve_opts;

/* Graph replay.  With graphs on, a batch of C cells of mechanism m and a
 * precision runs as one launch of a CUDA graph captured for (m, precision,
 * bucket), bucket = the power of two >= max(C, 256): the graph's kernels
 * (setup, max_iter x (Jacobian, Newton update), write-back) are bound to a
 * region of the arena that the graph keeps while it is cached, the batch's
 * inputs are copied there, and a device-side count tells the kernels how many
 * of the bucket's cells are real.  A bucket whose graph is busy on another
 * stream, or that does not fit next to the cached graphs, runs with direct
 * launches; idle graphs are released, least recently used first, when the
 * arena needs their memory.  Results are bit for bit those of direct
 * launches. */

typedef struct {
  uint64_t submitted, completed, rejected, queued, in_flight, batches, cells_completed;
  uint64_t bytes_in_use, bytes_peak;
  double p50_latency_us, p99_latency_us, mean_latency_us;  /* submit -> completion */
  double cells_per_s;   /* completed cells / (last completion - first submission) */
  uint64_t graph_batches;    /* batches run by replaying a captured graph */
  uint64_t graphs_captured;  /* graphs captured (a re-capture after release counts again) */
  uint64_t graphs_cached;    /* graphs held now */
  uint64_t in_flight_peak;   /* most batches on the device at once (streams in use) */
} qss_serve_stats_t;

int qss_serve_create(int device, size_t budget_bytes, const qss_serve_opts* opts, qss_server_t* out);
int qss_serve_submit(qss_server_t server, qss_mech_t mech, int64_t ncells, const double* rho,
                     double* T, double* Y, double dt, int precision, int32_t* iters,
                     int32_t* cell_status, uint64_t* req_id);
int qss_serve_wait(qss_server_t server, uint64_t req_id, int64_t timeout_us, int* req_status);
int qss_serve_stats(qss_server_t server, qss_serve_stats_t* out);
void qss_serve_destroy(qss_server_t server);

/* The implicit step for callers that cannot let the library allocate device
 * memory (the paper has no counterpart; this is a deployment variant).  Same
 * arguments, semantics and results as qss_implicit_step, but the Newton
 * scratch is a fixed 64 MiB array in the library's device memory instead of
 * memory the library allocates: applications that reserve and manage all of
 * the GPU's memory themselves, or loops that must not pay the synchronisation
 * an allocation can imply, call this one.  It calls no allocation routine; the
 * cells are processed in chunks that fit the array.  Every GPU that loads the
 * library holds the array until the process exits.  The first call on a device
 * looks up the array's device address (once per device, with that device
 * current), so make it before any stream capture.  Every call uses the same
 * array: two calls whose work overlaps on the GPU (different streams, or
 * different mechanism handles) race and corrupt each other; order them on one
 * stream.  The array keeps the last call's contents; each call initialises
 * every value it reads.  Errors: QSS_ERR_BUDGET if 32 cells of the mechanism
 * need more scratch than the array holds (the message gives both sizes). */
int qss_implicit_step_noalloc(qss_mech_t mech, int64_t ncells, int64_t ld, const double* dt,
                              int dt_stride, const double* rho, double* T, double* Y,
                              int precision, const qss_newton_opts* opts, int32_t* iters,
                              int32_t* cell_status, void* stream);

/* Message of the last failed call on the calling thread ("" if none). */
const char* qss_last_error(void);

/* Measured FP64 fused-multiply-add throughput of `device` in TFLOP/s
 * (2 flops per FMA), from a dependent-chain microbenchmark run for about
 * `millis` milliseconds.  Used as the FP64 roofline denominator. */
int qss_measure_fp64_peak(int device, int millis, double* tflops);

/* FP64 pipe probe (a measurement aid for kernel design; the paper has no
 * counterpart): one block of warps_per_sm warps on every SM, lanes running 8
 * FMAs per iteration as 8 independent chains (dependent = 0) or one dependent
 * chain (dependent = 1), with only active_lanes (32, 16, 8, 4 or 1) lanes of
 * each warp doing so.  *lane_tflops counts the active lanes' FMAs (2 flops
 * each); *cycles_per_warp_fma (nullable) is the SM sub-partition cycles per
 * warp-wide FMA instruction at the nominal clock.  On B300 a warp with 4
 * active lanes takes as long as a full one, and one warp per sub-partition
 * with a single dependent chain already keeps the pipe nearly busy. */
int qss_measure_fp64_pipe(int device, int warps_per_sm, int active_lanes, int dependent,
                          double* lane_tflops, double* cycles_per_warp_fma);

/* Diagnostics: evaluates the device math routines used by generated code,
 * elementwise on device arrays x[n] -> y[n] (fn 0 = table-driven exp,
 * 1 = CUDA library exp, 2 = table-driven log, 3 = series-refined reciprocal,
 * 4 = CUDA library log, 5 = CUDA correctly rounded reciprocal).  Used by the
 * tests that compare these functions with the library and with exact values.  Errors: QSS_ERR_INVALID_ARG for an
 * unknown fn or null arrays. */
int qss_selftest_math(int device, int fn, int64_t n, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QSS_H */

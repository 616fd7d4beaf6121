// Serving loop: continuous batching of implicit-step requests on one GPU.
//
// Requests (a mechanism, a batch of cells in host arrays, dt, a precision)
// are queued by qss_serve_submit.  A scheduler thread admits them as device
// memory and a stream slot become free, merging queued requests of the same
// mechanism and precision (in arrival order) into one launch of up to
// max_batch_cells cells.  Each admitted batch owns a region of a device arena
// whose size is the server's memory budget (this is the admission control:
// a batch waits until its inputs, outputs and Newton scratch fit), and one of
// n_streams streams, so batches overlap on the device.  Completion is
// detected with an event per batch; results land in the requests' host arrays
// (T and Y updated in place), and the latency submit -> completion is
// recorded.  A batch replays a CUDA graph captured for its (mechanism,
// precision, size bucket) when one is cached and idle (see qss.h).  Mechanism artefacts stay loaded (their constants are in the
// cubins); nothing is re-uploaded per request.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "qss_driver.h"
#include "qss_internal.h"

using namespace qss;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id;
  qss_mech_s* mech;
  int64_t ncells;
  const double* rho;
  double* T;
  double* Y;
  double dt;
  int precision;
  int32_t* iters;
  int32_t* status;
  Clock::time_point t_submit, t_done;
  int state = 0;   // 0 queued, 1 in flight, 2 done, 3 failed
  int rc = QSS_OK;
};

struct GraphEntry;

struct Batch {
  std::vector<Request*> reqs;
  int slot = -1;
  size_t off = 0, bytes = 0;
  int64_t cells = 0;
  GraphEntry* graph = nullptr;   // replayed graph (its own region), or direct launches
};

// A captured implicit step for (mechanism, precision, bucket): the graph and
// the arena region its kernels are bound to.
struct GraphEntry {
  CUgraphExec exec = nullptr;
  size_t off = 0, bytes = 0;
  int64_t bucket = 0;
  bool busy = false;
  uint64_t last_use = 0;
};
using GraphKey = std::tuple<qss_mech_s*, int, int64_t>;

// First-fit allocator over [0, size) of the device arena, 256-byte granules.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  size_t size_, used_ = 0;
  std::map<size_t, size_t> free_;
};

size_t batch_bytes(const qss_mech_s* m, int64_t cells, int precision, bool reuse, size_t* scratch_off) {
  const size_t c = (size_t)((cells + 31) / 32 * 32);
  size_t io = c * sizeof(double) * (3 + m->N) + c * 2 * sizeof(int32_t);   // rho, T, dt, Y; iters, status
  io = (io + 255) / 256 * 256;
  *scratch_off = io;
  return io + newton_scratch_per_cell(m, precision, reuse) * c + 256;
}

}  // namespace

struct qss_server_s {
  int device = 0;
  CUdevice dev = 0;
  CUcontext ctx = nullptr;
  CUdeviceptr arena_base = 0;
  Arena* arena = nullptr;
  int n_streams = 4;
  int64_t max_batch_cells = 1 << 18;
  qss_newton_opts newton;
  std::vector<CUstream> streams;
  std::vector<CUevent> events;
  std::vector<double*> pinned_dt;   // per-slot host staging of per-cell dt
  std::vector<size_t> pinned_cap;
  std::vector<Batch*> slot;         // batch in flight per slot (or null)
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  // stats
  std::vector<double> lat_us;
  uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, cells_done = 0;
  size_t bytes_peak = 0;
  Clock::time_point t_first, t_last;
  bool have_first = false;
  int fatal = QSS_OK;
  std::string fatal_msg;
  // graph replay
  bool graphs_on = true;
  std::map<GraphKey, GraphEntry> graphs;
  uint64_t use_clock = 0, graph_batches = 0, graphs_captured = 0;
  uint64_t in_flight_peak = 0;
};

namespace {

// Device layout of a batch region of `cap` cells (ldb = cap rounded to 32):
// rho, T, dt, Y[N] (doubles), iters, status (ints), then the Newton scratch at
// soff and, last, the int the capped kernels read as the real cell count.
struct Region {
  double *rho, *T, *dt, *Y;
  int32_t *it, *st;
  CUdeviceptr scratch;
  size_t scratch_bytes;
  int* ncap;
};

Region region_of(qss_server_s* s, qss_mech_s* m, size_t off, size_t bytes, int64_t cap, int prec,
                 bool with_count) {
  Region g;
  const size_t ldb = (size_t)((cap + 31) / 32 * 32);
  size_t soff;
  batch_bytes(m, cap, prec, s->newton.jac_reuse != 0, &soff);
  char* base = (char*)(s->arena_base + off);
  g.rho = (double*)base;
  g.T = g.rho + ldb;
  g.dt = g.T + ldb;
  g.Y = g.dt + ldb;
  g.it = (int32_t*)(g.Y + ldb * m->N);
  g.st = g.it + ldb;
  g.scratch = s->arena_base + off + soff;
  // a graph region carries 256 bytes more than batch_bytes: the cell count
  g.scratch_bytes = bytes - soff - (with_count ? 256 : 0);
  g.ncap = with_count ? (int*)(base + bytes - 256) : nullptr;
  return g;
}

int launch_batch(qss_server_s* s, Batch* b) {
  qss_mech_s* m = b->reqs[0]->mech;
  const int prec = b->reqs[0]->precision;
  const int64_t C = b->cells;
  const int64_t cap = b->graph ? b->graph->bucket : C;
  const size_t ldb = (size_t)((cap + 31) / 32 * 32);
  CUstream st = s->streams[b->slot];
  Region g = b->graph ? region_of(s, m, b->graph->off, b->graph->bytes, cap, prec, true)
                      : region_of(s, m, b->off, b->bytes, cap, prec, false);
  // per-cell dt staged in pinned host memory owned by the slot
  if (s->pinned_cap[b->slot] < (size_t)C) {
    if (s->pinned_dt[b->slot]) drv().cuMemFreeHost(s->pinned_dt[b->slot]);
    void* p = nullptr;
    CU_TRY(drv().cuMemHostAlloc(&p, (size_t)C * sizeof(double), 0));
    s->pinned_dt[b->slot] = (double*)p;
    s->pinned_cap[b->slot] = (size_t)C;
  }
  double* hdt = s->pinned_dt[b->slot];
  int64_t off = 0;
  for (Request* r : b->reqs) {
    for (int64_t i = 0; i < r->ncells; ++i) hdt[off + i] = r->dt;
    const size_t w = (size_t)r->ncells * sizeof(double);
    CU_TRY(drv().cuMemcpyHtoDAsync((CUdeviceptr)(g.rho + off), r->rho, w, st));
    CU_TRY(drv().cuMemcpyHtoDAsync((CUdeviceptr)(g.T + off), r->T, w, st));
    CUDA_MEMCPY2D c;
    std::memset(&c, 0, sizeof(c));
    c.srcMemoryType = CU_MEMORYTYPE_HOST;
    c.srcHost = r->Y;
    c.srcPitch = w;
    c.dstMemoryType = CU_MEMORYTYPE_DEVICE;
    c.dstDevice = (CUdeviceptr)(g.Y + off);
    c.dstPitch = ldb * sizeof(double);
    c.WidthInBytes = w;
    c.Height = m->N;
    CU_TRY(drv().cuMemcpy2DAsync(&c, st));
    off += r->ncells;
  }
  CU_TRY(drv().cuMemcpyHtoDAsync((CUdeviceptr)g.dt, hdt, (size_t)C * sizeof(double), st));
  if (b->graph) {
    CU_TRY(drv().cuMemsetD32Async((CUdeviceptr)g.ncap, (unsigned)C, 1, st));
    CU_TRY(drv().cuGraphLaunch(b->graph->exec, st));
    s->graph_batches++;
  } else {
    int rc = implicit_launch(m, C, (int64_t)ldb, g.dt, 1, g.rho, g.T, g.Y, prec, s->newton, g.it, g.st,
                             st, g.scratch, g.scratch_bytes);
    if (rc) return rc;
  }
  off = 0;
  for (Request* r : b->reqs) {
    const size_t w = (size_t)r->ncells * sizeof(double);
    CU_TRY(drv().cuMemcpyDtoHAsync(r->T, (CUdeviceptr)(g.T + off), w, st));
    CUDA_MEMCPY2D c;
    std::memset(&c, 0, sizeof(c));
    c.srcMemoryType = CU_MEMORYTYPE_DEVICE;
    c.srcDevice = (CUdeviceptr)(g.Y + off);
    c.srcPitch = ldb * sizeof(double);
    c.dstMemoryType = CU_MEMORYTYPE_HOST;
    c.dstHost = r->Y;
    c.dstPitch = w;
    c.WidthInBytes = w;
    c.Height = m->N;
    CU_TRY(drv().cuMemcpy2DAsync(&c, st));
    if (r->iters)
      CU_TRY(drv().cuMemcpyDtoHAsync(r->iters, (CUdeviceptr)(g.it + off), r->ncells * sizeof(int32_t), st));
    if (r->status)
      CU_TRY(drv().cuMemcpyDtoHAsync(r->status, (CUdeviceptr)(g.st + off), r->ncells * sizeof(int32_t), st));
    off += r->ncells;
  }
  CU_TRY(drv().cuEventRecord(s->events[b->slot], st));
  return QSS_OK;
}

// Release idle cached graphs, least recently used first, until `bytes` can be
// allocated from the arena (or none is left).  Returns true with *off set.
bool arena_alloc(qss_server_s* s, size_t bytes, size_t* off) {
  while (!s->arena->alloc(bytes, off)) {
    auto victim = s->graphs.end();
    for (auto it = s->graphs.begin(); it != s->graphs.end(); ++it)
      if (!it->second.busy && (victim == s->graphs.end() || it->second.last_use < victim->second.last_use))
        victim = it;
    if (victim == s->graphs.end()) return false;
    drv().cuGraphExecDestroy(victim->second.exec);
    s->arena->release(victim->second.off, victim->second.bytes);
    s->graphs.erase(victim);
  }
  return true;
}

// The cached graph for a batch of `cells` cells, captured on `st` if needed;
// null when graphs are off, the bucket's graph is busy, or memory is short.
// Called by the scheduler with s->mu held (lk); a capture (max_iter x 2
// launches recorded, then instantiated) runs with the lock released, so that
// submit, wait and stats do not block behind it.  The entry is reserved busy
// with its arena region before the lock is dropped: nothing else uses, evicts
// or captures it meanwhile (only the scheduler thread touches the graph cache
// and the arena, and `st` is the free slot's stream, used by no one else).
GraphEntry* graph_for(qss_server_s* s, qss_mech_s* m, int prec, int64_t cells, CUstream st,
                      std::unique_lock<std::mutex>& lk) {
  if (!s->graphs_on) return nullptr;
  int64_t bucket = 256;
  while (bucket < cells) bucket *= 2;
  if (bucket > s->max_batch_cells) return nullptr;
  GraphKey key(m, prec, bucket);
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    if (it->second.busy) return nullptr;
    it->second.last_use = ++s->use_clock;
    return &it->second;
  }
  size_t soff;
  const size_t bytes = batch_bytes(m, bucket, prec, s->newton.jac_reuse != 0, &soff) + 256;   // + the cell-count int
  size_t off;
  if (!arena_alloc(s, bytes, &off)) return nullptr;
  Region g = region_of(s, m, off, bytes, bucket, prec, true);
  const size_t ldb = (size_t)((bucket + 31) / 32 * 32);
  {
    GraphEntry& e = s->graphs[key];   // placeholder: busy, no executable yet
    e.exec = nullptr;
    e.off = off;
    e.bytes = bytes;
    e.bucket = bucket;
    e.busy = true;
    e.last_use = ++s->use_clock;
  }
  const qss_newton_opts newton = s->newton;
  lk.unlock();
  CUgraph graph = nullptr;
  CUgraphExec exec = nullptr;
  bool ok = drv().cuStreamBeginCapture(st, CU_STREAM_CAPTURE_MODE_RELAXED) == CUDA_SUCCESS;
  int rc = ok ? implicit_launch(m, bucket, (int64_t)ldb, g.dt, 1, g.rho, g.T, g.Y, prec, newton,
                                g.it, g.st, st, g.scratch, g.scratch_bytes, g.ncap)
              : QSS_ERR_CUDA;
  if (ok) ok = drv().cuStreamEndCapture(st, &graph) == CUDA_SUCCESS && rc == QSS_OK && graph;
  if (ok) ok = drv().cuGraphInstantiate(&exec, graph, 0) == CUDA_SUCCESS;
  if (graph) drv().cuGraphDestroy(graph);
  lk.lock();
  auto e = s->graphs.find(key);
  if (!ok) {
    s->arena->release(off, bytes);
    s->graphs.erase(e);
    return nullptr;
  }
  e->second.exec = exec;
  s->graphs_captured++;
  return &e->second;
}

void finish_batch(qss_server_s* s, Batch* b, int rc) {
  auto now = Clock::now();
  for (Request* r : b->reqs) {
    r->t_done = now;
    r->state = rc ? 3 : 2;
    r->rc = rc;
    if (!rc) {
      s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
      s->completed++;
      s->cells_done += r->ncells;
    }
  }
  s->t_last = now;
  if (b->graph)
    b->graph->busy = false;
  else
    s->arena->release(b->off, b->bytes);
  s->slot[b->slot] = nullptr;
  delete b;
}

void scheduler(qss_server_s* s) {
  drv().cuCtxSetCurrent(s->ctx);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // 1. completions
    bool any_inflight = false;
    for (size_t k = 0; k < s->slot.size(); ++k) {
      Batch* b = s->slot[k];
      if (!b) continue;
      CUresult q = drv().cuEventQuery(s->events[k]);
      if (q == CUDA_SUCCESS) {
        finish_batch(s, b, QSS_OK);
        s->cv_done.notify_all();
      } else if (q != CUDA_ERROR_NOT_READY) {
        finish_batch(s, b, QSS_ERR_CUDA);
        s->cv_done.notify_all();
      } else {
        any_inflight = true;
      }
    }
    if (s->stop && s->queue.empty() && !any_inflight) break;
    // 2. admission (arrival order; same mechanism and precision merged)
    while (!s->queue.empty()) {
      int free_slot = -1;
      for (size_t k = 0; k < s->slot.size(); ++k)
        if (!s->slot[k]) { free_slot = (int)k; break; }
      if (free_slot < 0) break;
      Request* head = s->queue.front();
      Batch* b = new Batch();
      b->reqs.push_back(head);
      b->cells = head->ncells;
      for (Request* r : s->queue) {
        if (r == head) continue;
        if (r->mech == head->mech && r->precision == head->precision &&
            b->cells + r->ncells <= s->max_batch_cells) {
          b->reqs.push_back(r);
          b->cells += r->ncells;
        }
      }
      // a cached (or newly captured) graph for the batch's size bucket, else
      // device memory for direct launches: shrink the batch (never below the
      // head request) until it fits, else wait for running batches
      size_t soff, need = 0;
      bool got = false;
      b->graph = graph_for(s, head->mech, head->precision, b->cells, s->streams[free_slot], lk);
      if (b->graph) {
        got = true;
        b->graph->busy = true;
      } else {
        while (true) {
          need = batch_bytes(head->mech, b->cells, head->precision, s->newton.jac_reuse != 0, &soff);
          if (arena_alloc(s, need, &b->off)) { got = true; break; }
          if (b->reqs.size() == 1) break;
          b->cells -= b->reqs.back()->ncells;
          b->reqs.pop_back();
        }
      }
      if (!got) {
        delete b;
        break;
      }
      b->bytes = need;
      b->slot = free_slot;
      s->slot[free_slot] = b;
      for (Request* r : b->reqs) {
        r->state = 1;
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
      }
      s->batches++;
      s->bytes_peak = std::max(s->bytes_peak, s->arena->used());
      {
        uint64_t busy = 0;
        for (Batch* x : s->slot) busy += x ? 1 : 0;
        s->in_flight_peak = std::max(s->in_flight_peak, busy);
      }
      int rc = launch_batch(s, b);
      if (rc) {
        s->fatal = rc;
        s->fatal_msg = g_err;
        drv().cuStreamSynchronize(s->streams[free_slot]);
        finish_batch(s, b, rc);
        s->cv_done.notify_all();
      }
    }
    // 3. sleep until new work or a short poll interval for completions
    s->cv_sched.wait_for(lk, std::chrono::microseconds(any_inflight ? 50 : 2000));
  }
}

}  // namespace

extern "C" {

int qss_serve_create(int device, size_t budget_bytes, const qss_serve_opts* opts, qss_server_t* out) {
  if (!out || budget_bytes < (size_t(1) << 20)) return fail(QSS_ERR_INVALID_ARG, "bad arguments");
  *out = nullptr;
  qss_server_s* s = new qss_server_s();
  int rc = ctx_for_device(device, &s->dev, &s->ctx);
  if (rc) { delete s; return rc; }
  s->device = device;
  s->newton = {20, 1e-12, 1e-20, 1e-10, 10, 1e-8, 0};
  if (opts) {
    if (opts->n_streams > 0) s->n_streams = opts->n_streams;
    if (opts->max_batch_cells > 0) s->max_batch_cells = opts->max_batch_cells;
    if (opts->newton) s->newton = *opts->newton;
    if (opts->graphs < 0) s->graphs_on = false;
  }
  CUresult r = drv().cuMemAlloc(&s->arena_base, budget_bytes);
  if (r != CUDA_SUCCESS) {
    drv().cuDevicePrimaryCtxRelease(s->dev);
    delete s;
    return fail(QSS_ERR_OOM, "cannot allocate the serving arena (budget)");
  }
  s->arena = new Arena(budget_bytes);
  for (int k = 0; k < s->n_streams; ++k) {
    CUstream st;
    CUevent ev;
    drv().cuStreamCreate(&st, CU_STREAM_NON_BLOCKING);
    drv().cuEventCreate(&ev, CU_EVENT_DISABLE_TIMING);
    s->streams.push_back(st);
    s->events.push_back(ev);
    s->slot.push_back(nullptr);
    s->pinned_dt.push_back(nullptr);
    s->pinned_cap.push_back(0);
  }
  s->worker = std::thread(scheduler, s);
  *out = s;
  return QSS_OK;
}

int qss_serve_submit(qss_server_t s, qss_mech_t mech, int64_t ncells, const double* rho, double* T,
                     double* Y, double dt, int precision, int32_t* iters, int32_t* cell_status,
                     uint64_t* req_id) {
  if (!s || !mech || !req_id) return fail(QSS_ERR_INVALID_ARG, "null argument");
  if (ncells <= 0 || !rho || !T || !Y) return fail(QSS_ERR_INVALID_ARG, "bad request arrays");
  if (precision != QSS_LU_FP64 && precision != QSS_LU_FP32_IR && precision != QSS_LU_MIXED)
    return fail(QSS_ERR_INVALID_ARG, "unknown precision");
  if (!(dt > 0)) return fail(QSS_ERR_INVALID_ARG, "dt must be positive");
  if (mech->ctx != s->ctx) return fail(QSS_ERR_INVALID_ARG, "mechanism loaded on another device");
  if (!mech->f_newton[lu_kind(precision)]) return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no Newton kernels");
  if (precision == QSS_LU_MIXED && !mech->jac32)
    return fail(QSS_ERR_UNIMPLEMENTED, "artefact has no mixed-precision Jacobian (jac32)");
  size_t soff;
  if (batch_bytes(mech, ncells, precision, s->newton.jac_reuse != 0, &soff) > s->arena->size() ||
      ncells > s->max_batch_cells) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->rejected++;
    return fail(QSS_ERR_BUDGET, "request larger than the server's memory budget or batch limit");
  }
  Request* r = new Request();
  r->mech = mech;
  r->ncells = ncells;
  r->rho = rho;
  r->T = T;
  r->Y = Y;
  r->dt = dt;
  r->precision = precision;
  r->iters = iters;
  r->status = cell_status;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    s->submitted++;
    if (!s->have_first) { s->t_first = r->t_submit; s->have_first = true; }
  }
  s->cv_sched.notify_one();
  *req_id = r->id;
  return QSS_OK;
}

int qss_serve_wait(qss_server_t s, uint64_t req_id, int64_t timeout_us, int* req_status) {
  if (!s) return fail(QSS_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return fail(QSS_ERR_INVALID_ARG, "unknown request id");
  Request* r = it->second;
  auto done = [&] { return r->state >= 2; };
  if (timeout_us < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    if (req_status) *req_status = QSS_ERR_TIMEOUT;
    return fail(QSS_ERR_TIMEOUT, "request not finished within the timeout");
  }
  int rc = r->rc;
  if (req_status) *req_status = rc;
  s->reqs.erase(it);
  delete r;
  return rc ? fail(rc, "request failed: " + s->fatal_msg) : QSS_OK;
}

int qss_serve_stats(qss_server_t s, qss_serve_stats_t* out) {
  if (!s || !out) return fail(QSS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->queued = s->queue.size();
  for (Batch* b : s->slot) out->in_flight += b ? b->reqs.size() : 0;
  out->batches = s->batches;
  out->cells_completed = s->cells_done;
  out->bytes_in_use = s->arena->used();
  out->bytes_peak = s->bytes_peak;
  out->graph_batches = s->graph_batches;
  out->graphs_captured = s->graphs_captured;
  out->graphs_cached = s->graphs.size();
  out->in_flight_peak = s->in_flight_peak;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    out->p50_latency_us = q(0.50);
    out->p99_latency_us = q(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_latency_us = sum / v.size();
  }
  if (s->have_first && s->completed) {
    double el = std::chrono::duration<double>(s->t_last - s->t_first).count();
    out->cells_per_s = el > 0 ? s->cells_done / el : 0.0;
  }
  return QSS_OK;
}

void qss_serve_destroy(qss_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->worker.joinable()) s->worker.join();
  drv().cuCtxSetCurrent(s->ctx);
  for (size_t k = 0; k < s->streams.size(); ++k) {
    drv().cuStreamSynchronize(s->streams[k]);
    drv().cuStreamDestroy(s->streams[k]);
    drv().cuEventDestroy(s->events[k]);
    if (s->pinned_dt[k]) drv().cuMemFreeHost(s->pinned_dt[k]);
  }
  for (auto& kv : s->reqs) delete kv.second;
  for (auto& kv : s->graphs) drv().cuGraphExecDestroy(kv.second.exec);
  drv().cuMemFree(s->arena_base);
  delete s->arena;
  drv().cuDevicePrimaryCtxRelease(s->dev);
  delete s;
}

}  // extern "C"

// Request server: continuous batching of independent least-squares solves
// on one device.
//
// Each request (A, b, options) is admitted when a slot is free and its HBM
// footprint (A, b and x, 256-byte aligned) fits in the server's device arena;
// A and b are then copied into the arena and the solve runs on that slot's
// own stream with a plan sized for (m_max, n_max).  Requests that arrive while
// others are on the GPU queue until a slot and memory free up, and the slots'
// kernels overlap on the device.  Admission is first come, first served (the
// head of the queue waits for memory rather than being overtaken).
//
// Each slot is driven by its own host thread: a solve waits on its stream a
// few times (after the QR for condest, during the step-1 stop test), and with
// one thread per slot those waits do not hold up the other slots.  The QR
// runs as one ordinary launch per column (no cooperative launch) so that
// concurrent solves cannot wait on each other's grid barriers.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <chrono>

#include "lsq_common.cuh"

using namespace lsq;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  lsq_options opt{};
  int method = 0;
  const double *A = nullptr, *b = nullptr;
  bool on_device = false;
  size_t off = 0, bytes = 0;
  lsq_status status = LSQ_PENDING;
  std::string err;
  lsq_info info{};
  std::vector<double> x;
  bool done = false;
  double t_submit = 0, t_start = 0, t_end = 0;
};

// First-fit allocator over [0, size) with coalescing free list.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t *off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t noff = it->first + bytes;
        free_.erase(it);
        if (rest) free_[noff] = rest;
        used_ += bytes;
        if (used_ > peak_) peak_ = used_;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
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
    used_ -= bytes;
  }
  size_t size() const { return size_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

}  // namespace

struct lsq_server_s {
  int dev = 0;
  char *arena_base = nullptr;
  Arena *arena = nullptr;
  int64_t m_max = 0, n_max = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, Request *> reqs;
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0, running = 0;
  bool stopping = false;
  struct Slot {
    cudaStream_t s = nullptr;
    lsq_plan plan = nullptr;      // slot mode: one solve at a time
    lsq_batch batch = nullptr;    // batch mode: up to max_batch solves per lockstep batch
    std::thread th;
  };
  std::vector<Slot> slots;
  int max_batch = 0;              // > 0: batch mode
  int64_t batch_elems = 0;        // plane capacity of each worker's batch engine
};

namespace {

size_t footprint(const lsq_options &o) {
  return align_up(sizeof(double) * (size_t)o.m * (size_t)o.n) + align_up(sizeof(double) * o.m) +
         align_up(sizeof(double) * o.n);
}

// Runs one request on the slot.  Returns false when the slot's stream could
// not be drained: the arena region may then still be read or written by work
// in flight, so the caller must not hand it to another request.
bool run_request(lsq_server S, lsq_server_s::Slot &slot, Request *r) {
  double *base = reinterpret_cast<double *>(S->arena_base + r->off);
  const size_t mn = (size_t)r->opt.m * r->opt.n;
  double *dA = base;
  double *db = reinterpret_cast<double *>(reinterpret_cast<char *>(dA) + align_up(sizeof(double) * mn));
  double *dx = reinterpret_cast<double *>(reinterpret_cast<char *>(db) +
                                          align_up(sizeof(double) * r->opt.m));
  const cudaMemcpyKind kind = r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(dA, r->A, sizeof(double) * mn, kind, slot.s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(db, r->b, sizeof(double) * r->opt.m, kind, slot.s);
  lsq_status st;
  if (e != cudaSuccess) {
    st = LSQ_ERR_CUDA;
    r->err = cudaGetErrorString(e);
  } else {
    lsq_options o = r->opt;
    o.lda = 0;
    st = plan_configure(slot.plan, &o);
    if (st >= 0) st = plan_solve(slot.plan, r->method, dA, db, dx, &r->info);
    if (st < 0) r->err = lsq_last_error();
  }
  if (st >= 0) {
    r->x.resize(r->opt.n);
    e = cudaMemcpyAsync(r->x.data(), dx, sizeof(double) * r->opt.n, cudaMemcpyDeviceToHost, slot.s);
    if (e != cudaSuccess) {
      st = LSQ_ERR_CUDA;
      r->err = cudaGetErrorString(e);
    }
  }
  // Whatever the status, nothing queued on the slot's stream may outlive the
  // request: an error can leave copies or kernels that read the region
  // behind it.
  e = cudaStreamSynchronize(slot.s);
  if (e != cudaSuccess && st >= 0) {
    st = LSQ_ERR_CUDA;
    r->err = cudaGetErrorString(e);
  }
  r->status = st;
  return e == cudaSuccess;
}

// Batch mode: copy the requests' A and b into their arena regions, solve
// them as one lockstep batch on the worker's engine, copy each x back.
// Returns false when the worker's stream could not be drained (the regions
// may still be in use and are not released).
bool run_batch(lsq_server S, lsq_server_s::Slot &slot, std::vector<Request *> &rs) {
  std::vector<lsq_batch_item> items(rs.size());
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < rs.size(); k++) {
    Request *r = rs[k];
    double *dA = reinterpret_cast<double *>(S->arena_base + r->off);
    const size_t mn = (size_t)r->opt.m * r->opt.n;
    double *db = reinterpret_cast<double *>(reinterpret_cast<char *>(dA) + align_up(sizeof(double) * mn));
    double *dx = reinterpret_cast<double *>(reinterpret_cast<char *>(db) +
                                            align_up(sizeof(double) * r->opt.m));
    const cudaMemcpyKind kind = r->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dA, r->A, sizeof(double) * mn, kind, slot.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, r->b, sizeof(double) * r->opt.m, kind, slot.s);
    items[k].m = r->opt.m;
    items[k].n = r->opt.n;
    items[k].A = dA;
    items[k].b = db;
    items[k].x = dx;
    items[k].seed = r->opt.seed;
    items[k].method = r->method;
    items[k].status = 0;
  }
  std::vector<lsq_info> infos(rs.size());
  lsq_status st = LSQ_OK;
  std::string err;
  if (e != cudaSuccess) {
    st = LSQ_ERR_CUDA;
    err = cudaGetErrorString(e);
  } else {
    st = lsq_batch_solve(slot.batch, (int)rs.size(), items.data(), infos.data());
    if (st < 0) err = lsq_last_error();
  }
  // an error of the call itself (copies, launches) fails every item; an
  // error of some items (non-finite data, zero column) only those
  bool item_error = false;
  for (const lsq_batch_item &q : items) item_error = item_error || q.status < 0;
  const bool call_failed = st < 0 && !item_error;
  for (size_t k = 0; k < rs.size(); k++) {
    Request *r = rs[k];
    const lsq_status sk = call_failed ? st : (lsq_status)items[k].status;
    r->status = sk;
    r->info = infos[k];
    r->info.status = sk;
    if (sk >= 0) {
      r->x.resize(r->opt.n);
      cudaError_t ex = cudaMemcpyAsync(r->x.data(), items[k].x, sizeof(double) * r->opt.n,
                                       cudaMemcpyDeviceToHost, slot.s);
      if (ex != cudaSuccess) {
        r->status = LSQ_ERR_CUDA;
        r->err = cudaGetErrorString(ex);
      }
    } else {
      r->err = err.empty() ? "the item failed in its batch" : err;
    }
  }
  e = cudaStreamSynchronize(slot.s);
  if (e != cudaSuccess)
    for (Request *r : rs)
      if (r->status >= 0) {
        r->status = LSQ_ERR_CUDA;
        r->err = cudaGetErrorString(e);
      }
  return e == cudaSuccess;
}

int64_t plane_elems(const lsq_options &o) { return o.m * ((o.n + 3) / 4 * 4); }

void batch_worker(lsq_server S, int idx) {
  cudaSetDevice(S->dev);
  lsq_server_s::Slot &slot = S->slots[idx];
  for (;;) {
    std::vector<Request *> rs;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stopping) return;
        // first come, first served: take requests from the head while the
        // batch, the worker's planes and the arena have room
        int64_t elems = 0;
        while (!S->queue.empty() && (int)rs.size() < S->max_batch) {
          Request *r = S->queue.front();
          if (elems + plane_elems(r->opt) > S->batch_elems) break;
          if (!S->arena->alloc(r->bytes, &r->off)) break;
          elems += plane_elems(r->opt);
          rs.push_back(r);
          S->queue.pop_front();
          S->running++;
        }
        if (!rs.empty()) break;
        S->cv.wait(lk);
      }
    }
    const double t0 = now_s();
    for (Request *r : rs) r->t_start = t0;
    const bool drained = run_batch(S, slot, rs);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const double t1 = now_s();
      for (Request *r : rs) {
        if (drained) S->arena->release(r->off, r->bytes);
        r->t_end = t1;
        r->done = true;
        S->running--;
        S->completed++;
      }
    }
    S->cv.notify_all();
  }
}

void worker(lsq_server S, int idx) {
  cudaSetDevice(S->dev);
  lsq_server_s::Slot &slot = S->slots[idx];
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stopping) return;
        if (!S->queue.empty() && S->arena->alloc(S->queue.front()->bytes, &S->queue.front()->off)) {
          r = S->queue.front();
          S->queue.pop_front();
          S->running++;
          break;
        }
        S->cv.wait(lk);
      }
    }
    r->t_start = now_s();
    const bool drained = run_request(S, slot, r);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      // a region whose stream could not be drained stays allocated (leaked
      // for the server's lifetime) rather than being handed out again
      if (drained) S->arena->release(r->off, r->bytes);
      r->t_end = now_s();
      r->done = true;
      S->running--;
      S->completed++;
    }
    S->cv.notify_all();
  }
}

void destroy_server(lsq_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv.notify_all();
  for (auto &sl : S->slots)
    if (sl.th.joinable()) sl.th.join();
  for (auto &sl : S->slots) {
    if (sl.plan) lsq_plan_destroy(sl.plan);
    if (sl.batch) lsq_batch_destroy(sl.batch);
    if (sl.s) cudaStreamDestroy(sl.s);
  }
  for (auto &kv : S->reqs) delete kv.second;
  if (S->arena_base) cudaFree(S->arena_base);
  delete S->arena;
  delete S;
}

}  // namespace

extern "C" {

lsq_status lsq_server_create(size_t arena_bytes, int max_slots, int64_t m_max, int64_t n_max,
                             lsq_server *out) {
  if (!out) {
    set_last_error("out is NULL");
    return LSQ_ERR_INVALID;
  }
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64 || m_max < 1 || n_max < 1 || m_max < n_max ||
      n_max > LSQ_MAX_N || arena_bytes < kAlign) {
    set_last_error("need 1 <= max_slots <= 64, m_max >= n_max >= 1, n_max <= LSQ_MAX_N");
    return LSQ_ERR_INVALID;
  }
  lsq_server S = new lsq_server_s();
  S->m_max = m_max;
  S->n_max = n_max;
  cudaError_t e = cudaGetDevice(&S->dev);
  if (e == cudaSuccess) e = cudaMalloc((void **)&S->arena_base, arena_bytes);
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    set_last_error(cudaGetErrorString(e));
    destroy_server(S);
    return oom ? LSQ_ERR_OOM : LSQ_ERR_CUDA;
  }
  S->arena = new Arena(arena_bytes);
  S->slots.resize(max_slots);
  for (int i = 0; i < max_slots; i++) {
    e = cudaStreamCreateWithFlags(&S->slots[i].s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      destroy_server(S);
      return LSQ_ERR_CUDA;
    }
    lsq_options o;
    lsq_options_default(&o);
    o.m = m_max;
    o.n = n_max;
    lsq_status st = lsq_plan_create(&o, S->slots[i].s, &S->slots[i].plan);
    if (st < 0) {
      destroy_server(S);
      return st;
    }
    plan_set_stepwise_qr(S->slots[i].plan, 1);
  }
  for (int i = 0; i < max_slots; i++) S->slots[i].th = std::thread(worker, S, i);
  *out = S;
  return LSQ_OK;
}

lsq_status lsq_server_create_batched(size_t arena_bytes, int workers, int max_batch,
                                     int64_t m_max, int64_t n_max, lsq_server *out) {
  if (!out) {
    set_last_error("out is NULL");
    return LSQ_ERR_INVALID;
  }
  *out = nullptr;
  if (workers < 1 || workers > 8 || max_batch < 1 || max_batch > 256 || m_max < 1 ||
      n_max < 1 || m_max < n_max || n_max > 256 || arena_bytes < kAlign) {
    set_last_error("need 1 <= workers <= 8, 1 <= max_batch <= 256, m_max >= n_max >= 1, "
                   "n_max <= 256");
    return LSQ_ERR_INVALID;
  }
  lsq_server S = new lsq_server_s();
  S->m_max = m_max;
  S->n_max = n_max;
  S->max_batch = max_batch;
  // each worker's planes hold as many elements as the arena holds entries of
  // A, but never more than max_batch requests of the largest shape need
  const int64_t npad4 = (n_max + 3) / 4 * 4;
  S->batch_elems = std::max<int64_t>(
      std::min<int64_t>((int64_t)(arena_bytes / sizeof(double)), max_batch * m_max * npad4),
      m_max * npad4);
  cudaError_t e = cudaGetDevice(&S->dev);
  if (e == cudaSuccess) e = cudaMalloc((void **)&S->arena_base, arena_bytes);
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    set_last_error(cudaGetErrorString(e));
    destroy_server(S);
    return oom ? LSQ_ERR_OOM : LSQ_ERR_CUDA;
  }
  S->arena = new Arena(arena_bytes);
  S->slots.resize(workers);
  for (int i = 0; i < workers; i++) {
    e = cudaStreamCreateWithFlags(&S->slots[i].s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      set_last_error(cudaGetErrorString(e));
      destroy_server(S);
      return LSQ_ERR_CUDA;
    }
    lsq_status st = lsq_batch_create(max_batch, n_max, S->batch_elems, S->slots[i].s,
                                     &S->slots[i].batch);
    if (st < 0) {
      destroy_server(S);
      return st;
    }
  }
  for (int i = 0; i < workers; i++) S->slots[i].th = std::thread(batch_worker, S, i);
  *out = S;
  return LSQ_OK;
}

lsq_status lsq_submit(lsq_server S, const lsq_options *opt, int method, const double *A,
                      const double *b, int on_device, uint64_t *ticket) {
  if (!S || !opt || !A || !b || !ticket) {
    set_last_error("NULL argument");
    return LSQ_ERR_INVALID;
  }
  if (method < 0 || method > 2) {
    set_last_error("method must be 0 (FOSSILS), 1 (SPIR) or 2 (LSQR-based SPIR)");
    return LSQ_ERR_INVALID;
  }
  if (opt->m > S->m_max || opt->n > S->n_max || opt->n < 1 || opt->m < opt->n ||
      (opt->lda != 0 && opt->lda != opt->n) || opt->nrhs != 0 ||
      (opt->zeta != 0 && opt->zeta > 8) || (opt->d != 0 && opt->d > 12 * S->n_max) ||
      (opt->precision != LSQ_PREC_FP64)) {
    set_last_error("request outside the server's limits (m <= m_max, n <= n_max, lda = n, "
                   "zeta <= 8, d <= 12 n_max, FP64, one right-hand side)");
    return LSQ_ERR_INVALID;
  }
  if (S->max_batch > 0 && method == 2) {
    set_last_error("a batched server takes FOSSILS (0) and SPIR (1) requests");
    return LSQ_ERR_INVALID;
  }
  if (S->max_batch > 0 && plane_elems(*opt) > S->batch_elems) {
    set_last_error("request larger than a batch worker's planes");
    return LSQ_ERR_OOM;
  }
  Request *r = new Request();
  r->opt = *opt;
  r->method = method;
  r->A = A;
  r->b = b;
  r->on_device = on_device != 0;
  r->bytes = footprint(*opt);
  if (r->bytes > S->arena->size()) {
    delete r;
    set_last_error("request footprint exceeds the server arena");
    return LSQ_ERR_OOM;
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    S->submitted++;
  }
  S->cv.notify_all();
  *ticket = r->ticket;
  return LSQ_OK;
}

lsq_status lsq_poll(lsq_server S, uint64_t ticket, double *x, lsq_info *info, double *latency_s) {
  if (!S) {
    set_last_error("server is NULL");
    return LSQ_ERR_INVALID;
  }
  Request *r = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
      set_last_error("unknown ticket");
      return LSQ_ERR_INVALID;
    }
    if (!it->second->done) return LSQ_PENDING;
    r = it->second;
    S->reqs.erase(it);
  }
  const lsq_status st = r->status;
  if (st >= 0 && x) std::memcpy(x, r->x.data(), sizeof(double) * r->opt.n);
  if (info) *info = r->info;
  if (latency_s) *latency_s = r->t_end - r->t_submit;
  if (st < 0) set_last_error(r->err.c_str());
  delete r;
  return st;
}

lsq_status lsq_server_stats(lsq_server S, int64_t *out7) {
  if (!S || !out7) {
    set_last_error("NULL argument");
    return LSQ_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  out7[0] = S->submitted;
  out7[1] = S->completed;
  out7[2] = (int64_t)S->queue.size();
  out7[3] = S->running;
  out7[4] = (int64_t)S->arena->size();
  out7[5] = (int64_t)S->arena->used();
  out7[6] = (int64_t)S->arena->peak();
  return LSQ_OK;
}

void lsq_server_destroy(lsq_server S) { destroy_server(S); }

}  // extern "C"

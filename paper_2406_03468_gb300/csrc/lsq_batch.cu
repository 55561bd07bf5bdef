// Batched solves: many independent least-squares problems (n <= 256) solved
// in lockstep, every phase of the method one launch over all of them.
//
// A single FOSSILS / SPIR solve of a small problem is a few hundred short
// kernels (sketch, QR, setup, and five per inner update); for problems of
// 1e4..4e5 rows each kernel runs for microseconds, about the cost of its
// launch.  Here the problems of a batch share every launch: the sketch, each
// QR column step, the setup after the QR, and each refinement phase cover all
// items (one item per CTA for the n-vector work, the items' rows dealt over
// the CTAs of the streaming passes in proportion to m n).  Items whose inner
// loop has stopped (device-side flag, as on the single-problem path) return
// at once from the inner-loop kernels.  The launches of each phase are
// captured once in a CUDA graph and replayed.
//
// Per item the method is the plan path's (Alg. 1 with FOSSILS' Polyak or
// SPIR's CG, the rules of Sec. 4.2 / Alg. 4): column scaling, the sparse sign
// sketch (scatter form, FP64 atomics), Householder QR of the sketch (the
// stepwise form), condest / normest, x0, two refinement steps with the
// step-1 threshold and the q0 - 1 step-2 count.  The inner passes run in
// double-float on the item's hi / lo FP32 planes (written by the sketch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "lsq_common.cuh"

using namespace lsq;

namespace {

constexpr int kBatchNMax = 256;
constexpr int kBatchZeta = 8;
constexpr int kCondIters = 10;
constexpr int kPollEvery = 4;
constexpr uint64_t kQrTimeoutNs = 5ull * 1000 * 1000 * 1000;  // 5 s per inter-CTA wait

lsq_status bfail(lsq_status st, const std::string &msg) {
  set_last_error(msg.c_str());
  return st;
}

#define BCU(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return bfail(LSQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct lsq_batch_s {
  int dev = 0, nsm = 0;
  int max_items = 0;
  int64_t n_max = 0, elems_max = 0;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  // pools
  char *ws = nullptr;            // per-item n- and d-sized buffers
  size_t ws_per_item = 0;
  float *planes = nullptr;       // hi / lo planes of all items (elems_max floats each)
  double *part = nullptr, *r2part = nullptr;  // pass partials (per item: grid_max x 256)
  int grid_max = 0;
  DevState *st = nullptr;        // one per item
  BItem *d_items = nullptr;
  int *d_cta = nullptr;
  BItem *h_items = nullptr;      // pinned staging of the table
  int *h_cta = nullptr;
  int *d_qmap = nullptr, *h_qmap = nullptr;  // CTA -> item map of the batched QR
  int qgrid = 0;                 // CTAs of the batched QR (0: the column-step form)
  int qr_epoch = 0;              // flag value of the next batched QR
  DevState *h_st = nullptr;      // pinned copy of the states
  // captured phases, keyed by (count, grid, nmax)
  struct Graphs {
    cudaGraphExec_t pre = nullptr, setup = nullptr, step0 = nullptr, step1 = nullptr,
                    iter = nullptr, post = nullptr;
  };
  std::map<std::tuple<int, int, int>, Graphs> graphs;
  int grid = 0;                  // row-parallel CTAs of the current solve
};

namespace {

// Byte layout of one item's slice of the workspace.
struct Slice {
  size_t SAb, W, Rcm, Rrm, Dt, vhead, vec, qflag, total;
};

Slice slice_layout(int64_t nmax) {
  const size_t n = (size_t)nmax, d = 12 * n, nb = (n + 31) / 32;
  Slice L;
  size_t o = 0;
  L.SAb = o; o += a256(sizeof(double) * d * (n + 1));
  L.W = o; o += a256(sizeof(double) * d * (n + 1));
  L.Rcm = o; o += a256(sizeof(double) * n * n);
  L.Rrm = o; o += a256(sizeof(double) * n * n);
  L.Dt = o; o += a256(sizeof(double) * 2 * nb * 1024);
  L.vhead = o; o += a256(sizeof(double) * 2 * d);
  L.vec = o; o += a256(sizeof(double) * 17 * n);
  L.qflag = o; o += a256(sizeof(int) * (n + 1));
  L.total = o;
  return L;
}

// Autotuned row-parallel CTAs per SM for the streaming passes, keyed by the
// batch's shape class; measured once per process and class (b_resid over the
// batch at 1, 2 and 4 CTAs per SM), remembered in a text file when
// LSQ_AUTOTUNE_FILE names one (lines "nsm count_class mn_class ctas_per_sm").
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;
bool g_tune_loaded = false;

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char *path = std::getenv("LSQ_AUTOTUNE_FILE");
  if (!path) return;
  std::ifstream f(path);
  int a, b, c, v;
  while (f >> a >> b >> c >> v) g_tune[{a, b, c}] = v;
}

void tune_store(const std::tuple<int, int, int> &key, int v) {
  g_tune[key] = v;
  const char *path = std::getenv("LSQ_AUTOTUNE_FILE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << std::get<0>(key) << " " << std::get<1>(key) << " " << std::get<2>(key) << " " << v << "\n";
}

int log2_class(double v) {
  int c = 0;
  while (v >= 2.0 && c < 62) {
    v *= 0.5;
    c++;
  }
  return c;
}

// Deal `grid` CTAs to the items in proportion to m n (at least one each);
// fills cta0 / ncta of the table and the CTA -> item map.
void deal_ctas(lsq_batch B, int count, int grid) {
  double tot = 0.0;
  for (int i = 0; i < count; i++) tot += (double)B->h_items[i].m * B->h_items[i].n;
  std::vector<int> cnt(count, 1);
  int left = grid - count;
  std::vector<std::pair<double, int>> frac;
  for (int i = 0; i < count; i++) {
    const double share = (double)B->h_items[i].m * B->h_items[i].n / tot * left;
    const int f = (int)std::floor(share);
    cnt[i] += f;
    frac.push_back({share - f, i});
  }
  int used = 0;
  for (int c : cnt) used += c;
  std::sort(frac.begin(), frac.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
    return a.first > b.first;
  });
  for (size_t k = 0; k < frac.size() && used < grid; k++, used++) cnt[frac[k].second]++;
  int g = 0;
  for (int i = 0; i < count; i++) {
    B->h_items[i].cta0 = g;
    B->h_items[i].ncta = cnt[i];
    for (int c = 0; c < cnt[i]; c++) B->h_cta[g++] = i;
  }
}

}  // namespace

extern "C" {

lsq_status lsq_batch_create(int max_items, int64_t n_max, int64_t elems_max, void *cuda_stream,
                            lsq_batch *out) {
  if (!out) return bfail(LSQ_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (max_items < 1 || max_items > 256 || n_max < 1 || n_max > kBatchNMax || elems_max < n_max)
    return bfail(LSQ_ERR_INVALID, "need 1 <= max_items <= 256, 1 <= n_max <= 256, "
                                  "elems_max >= n_max");
  lsq_batch B = new lsq_batch_s();
  B->max_items = max_items;
  B->n_max = n_max;
  B->elems_max = elems_max;
  cudaError_t e = cudaGetDevice(&B->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, B->dev);
  if (e == cudaSuccess && cuda_stream == nullptr) {
    e = cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking);
    B->own_stream = true;
  } else {
    B->s = (cudaStream_t)cuda_stream;
  }
  const Slice L = slice_layout(n_max);
  B->ws_per_item = L.total;
  B->grid_max = std::max(4 * B->nsm, max_items);
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(cudaMalloc((void **)&B->ws, L.total * (size_t)max_items));
  A(cudaMalloc((void **)&B->planes, sizeof(float) * 2 * (size_t)elems_max + 256));
  // each item's partials hold a whole grid (the CTAs are re-dealt to the
  // unfinished items as the inner loop goes on)
  A(cudaMalloc((void **)&B->part, sizeof(double) * (size_t)max_items * B->grid_max * 256));
  A(cudaMalloc((void **)&B->r2part, sizeof(double) * (size_t)max_items * B->grid_max));
  A(cudaMalloc((void **)&B->st, sizeof(DevState) * (size_t)max_items));
  A(cudaMalloc((void **)&B->d_items, sizeof(BItem) * (size_t)max_items));
  A(cudaMalloc((void **)&B->d_cta, sizeof(int) * (size_t)B->grid_max));
  A(cudaMallocHost((void **)&B->h_items, sizeof(BItem) * (size_t)max_items));
  A(cudaMallocHost((void **)&B->h_cta, sizeof(int) * (size_t)B->grid_max));
  A(cudaMallocHost((void **)&B->h_st, sizeof(DevState) * (size_t)max_items));
  A(cudaMalloc((void **)&B->d_qmap, sizeof(int) * (size_t)b_qr_max_ctas(B->nsm)));
  A(cudaMallocHost((void **)&B->h_qmap, sizeof(int) * (size_t)b_qr_max_ctas(B->nsm)));
  // the QR flags start at 0 (a flag is ready when it equals the launch's epoch)
  if (e == cudaSuccess) A(cudaMemset(B->ws, 0, L.total * (size_t)max_items));
  A(prepare_b_kernels((int)n_max));
  A(prepare_b_inner());
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    lsq_batch_destroy(B);
    return bfail(oom ? LSQ_ERR_OOM : LSQ_ERR_CUDA, std::string("batch allocation: ") + cudaGetErrorString(e));
  }
  *out = B;
  return LSQ_OK;
}

void lsq_batch_destroy(lsq_batch B) {
  if (!B) return;
  if (B->s) cudaStreamSynchronize(B->s);
  for (auto &kv : B->graphs) {
    cudaGraphExec_t g[] = {kv.second.pre, kv.second.setup, kv.second.step0, kv.second.step1,
                           kv.second.iter, kv.second.post};
    for (auto x : g)
      if (x) cudaGraphExecDestroy(x);
  }
  void *bufs[] = {B->ws, B->planes, B->part, B->r2part, B->st, B->d_items, B->d_cta, B->d_qmap};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (B->h_items) cudaFreeHost(B->h_items);
  if (B->h_cta) cudaFreeHost(B->h_cta);
  if (B->h_st) cudaFreeHost(B->h_st);
  if (B->h_qmap) cudaFreeHost(B->h_qmap);
  if (B->own_stream && B->s) cudaStreamDestroy(B->s);
  delete B;
}

}  // extern "C"

namespace {

// Capture the launches `fn` makes on B->s into an executable graph.
template <class F>
lsq_status capture(lsq_batch B, cudaGraphExec_t *out, F fn) {
  cudaGraph_t g = nullptr;
  BCU(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = fn();
  cudaError_t e2 = cudaStreamEndCapture(B->s, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(LSQ_ERR_CUDA, std::string("graph capture: ") +
                                   cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(LSQ_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return LSQ_OK;
}

lsq_status read_states(lsq_batch B, int count) {
  BCU(cudaMemcpyAsync(B->h_st, B->st, sizeof(DevState) * (size_t)count, cudaMemcpyDeviceToHost,
                      B->s));
  BCU(cudaStreamSynchronize(B->s));
  return LSQ_OK;
}

}  // namespace

extern "C" lsq_status lsq_batch_solve(lsq_batch B, int count, lsq_batch_item *items,
                                      lsq_info *infos) {
  if (!B) return bfail(LSQ_ERR_INVALID, "batch is NULL");
  if (count < 1 || count > B->max_items || !items)
    return bfail(LSQ_ERR_INVALID, "need 1 <= count <= max_items and items");
  int nmax = 0;
  int64_t elems = 0;
  for (int i = 0; i < count; i++) {
    const lsq_batch_item &q = items[i];
    if (!q.A || !q.b || !q.x) return bfail(LSQ_ERR_INVALID, "item with a NULL pointer");
    if (q.n < 1 || q.n > B->n_max || q.m < q.n) return bfail(LSQ_ERR_INVALID, "item outside 1 <= n <= n_max, m >= n");
    if (q.method != 0 && q.method != 1) return bfail(LSQ_ERR_INVALID, "item method must be 0 or 1");
    nmax = std::max<int>(nmax, (int)q.n);
    elems += q.m * ((q.n + 3) / 4 * 4);
  }
  if (elems > B->elems_max) return bfail(LSQ_ERR_INVALID, "batch exceeds the plane capacity (elems_max)");
  // the table: sizes, pointers into the pools
  const Slice L = slice_layout(B->n_max);
  int64_t poff = 0;
  for (int i = 0; i < count; i++) {
    const lsq_batch_item &q = items[i];
    BItem &it = B->h_items[i];
    std::memset(&it, 0, sizeof(it));
    it.A = q.A;
    it.b = q.b;
    it.x = q.x;
    it.m = q.m;
    it.n = (int)q.n;
    it.npad = pass_npad(it.n);
    it.d = 12 * it.n;
    it.ld32 = (it.n + 3) / 4 * 4;
    it.method = q.method;
    it.seed = q.seed;
    it.eta = std::sqrt((double)it.n / (double)it.d);
    it.beta = it.eta * it.eta;
    it.alpha = (1.0 - it.beta) * (1.0 - it.beta);
    char *base = B->ws + B->ws_per_item * (size_t)i;
    it.SAb = (double *)(base + L.SAb);
    it.W = (double *)(base + L.W);
    it.Rcm = (double *)(base + L.Rcm);
    it.Rrm = (double *)(base + L.Rrm);
    it.Dt = (double *)(base + L.Dt);
    it.vhead = (double *)(base + L.vhead);
    double *v = (double *)(base + L.vec);
    const int64_t nm = B->n_max;
    double **vs[] = {&it.dcol, &it.dinv, &it.rinv, &it.t, &it.xs, &it.xo, &it.c, &it.g, &it.dy,
                     &it.dyold, &it.z, &it.h, &it.w, &it.res, &it.p};
    for (size_t k = 0; k < sizeof(vs) / sizeof(vs[0]); k++) *vs[k] = v + k * nm;
    it.Ahi = B->planes + poff;
    it.Alo = B->planes + B->elems_max + poff;
    poff += it.m * it.ld32;
    poff = (poff + 3) / 4 * 4;
    it.st = B->st + i;
    it.qflag = (int *)(base + L.qflag);
  }
  // QR groups: CTAs in proportion to d n^2, at least enough that no CTA holds
  // more than 32 columns; if the items need more CTAs than one cooperative
  // launch can hold, the QR takes the column-step form
  {
    const int qmax = b_qr_max_ctas(B->nsm);
    int need = 0;
    double work = 0.0;
    for (int i = 0; i < count; i++) {
      need += b_qr_min_ctas(B->h_items[i].n);
      work += (double)B->h_items[i].d * B->h_items[i].n * B->h_items[i].n;
    }
    B->qgrid = 0;
    if (need <= qmax) {
      int g = 0;
      const int spare = qmax - need;
      for (int i = 0; i < count; i++) {
        BItem &it = B->h_items[i];
        const double share = (double)it.d * it.n * it.n / work;
        int c = b_qr_min_ctas(it.n) + (int)std::floor(share * spare);
        c = std::min(c, it.n + 1);  // no more CTAs than columns
        it.qcta0 = g;
        it.qncta = c;
        for (int k = 0; k < c; k++) B->h_qmap[g + k] = i;
        g += c;
      }
      B->qgrid = g;
    }
  }
  // row-parallel CTAs: autotuned per shape class (1, 2 or 4 per SM)
  double mn = 0.0;
  for (int i = 0; i < count; i++) mn += (double)items[i].m * items[i].n;
  const std::tuple<int, int, int> key{B->nsm, log2_class(count), log2_class(mn)};
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load();
    auto f = g_tune.find(key);
    if (f != g_tune.end()) per_sm = f->second;
  }
  auto set_grid = [&](int ps) -> lsq_status {
    B->grid = std::max(ps * B->nsm, count);
    B->grid = std::min(B->grid, B->grid_max);
    deal_ctas(B, count, B->grid);
    for (int i = 0; i < count; i++) {
      BItem &it = B->h_items[i];
      it.part = B->part + (size_t)i * B->grid_max * 256;
      it.r2part = B->r2part + (size_t)i * B->grid_max;
    }
    BCU(cudaMemcpyAsync(B->d_items, B->h_items, sizeof(BItem) * count, cudaMemcpyHostToDevice, B->s));
    BCU(cudaMemcpyAsync(B->d_cta, B->h_cta, sizeof(int) * B->grid, cudaMemcpyHostToDevice, B->s));
    if (B->qgrid > 0)
      BCU(cudaMemcpyAsync(B->d_qmap, B->h_qmap, sizeof(int) * B->qgrid, cudaMemcpyHostToDevice,
                          B->s));
    return LSQ_OK;
  };
  // the partials hold grid x 256 doubles: fits for any deal (npad <= 256)
  BCU(cudaMemsetAsync(B->st, 0, sizeof(DevState) * (size_t)count, B->s));
  const int qcta = std::max(1, std::min(8, 2 * B->nsm / count));
  // sketch (and, when the QR takes the column-step form, the QR steps)
  const bool coop_qr = B->qgrid > 0;
  auto pre = [&]() -> cudaError_t {
    cudaError_t e = launch_b_zero(B->d_items, count, B->s);
    if (e == cudaSuccess) e = launch_b_sketch(B->d_items, B->d_cta, B->grid, kBatchZeta, B->s);
    if (e == cudaSuccess) e = launch_b_finalize(B->d_items, count, kBatchZeta, B->s);
    for (int k = -1; !coop_qr && k < nmax && e == cudaSuccess; k++)
      e = launch_b_qr_step(B->d_items, count, qcta, k, B->s);
    return e;
  };
  auto setup = [&]() -> cudaError_t {
    return launch_b_setup(B->d_items, count, kCondIters, 100, nmax, B->s);
  };
  if (per_sm == 0) {
    // tune: time the residual pass over this batch (it only writes partials,
    // which the solve overwrites) at 1, 2 and 4 CTAs per SM, with x = 0: the
    // same traffic as in the solve
    for (int i = 0; i < count; i++)
      BCU(cudaMemsetAsync(B->h_items[i].dcol, 0, sizeof(double) * 17 * (size_t)B->n_max, B->s));
    float best = 1e30f;
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    for (int ps : {1, 2, 4}) {
      if (ps * B->nsm > B->grid_max) continue;
      lsq_status st = set_grid(ps);
      if (st < 0) return st;
      BCU(launch_b_resid(B->d_items, B->d_cta, B->grid, B->s));  // warm
      BCU(cudaEventRecord(e0, B->s));
      BCU(launch_b_resid(B->d_items, B->d_cta, B->grid, B->s));
      BCU(cudaEventRecord(e1, B->s));
      BCU(cudaStreamSynchronize(B->s));
      float ms = 0.f;
      BCU(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        per_sm = ps;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store(key, per_sm);
  }
  {
    lsq_status st = set_grid(per_sm);
    if (st < 0) return st;
  }
  // phases, captured once per (count, grid, nmax) and replayed
  auto &G = B->graphs[{count, B->grid, nmax * 2 + (coop_qr ? 1 : 0)}];
  if (!G.pre) {
    lsq_status st = capture(B, &G.pre, pre);
    if (st < 0) return st;
    st = capture(B, &G.setup, setup);
    if (st < 0) return st;
    const double gam = 10.0, rho = 0.4;  // Alg. 4's step-1 stop constants
    for (int step = 0; step < 2; step++) {
      st = capture(B, step == 0 ? &G.step0 : &G.step1, [&]() -> cudaError_t {
        cudaError_t e = launch_b_redeal(B->d_items, count, B->d_cta, B->grid, 1, B->s);
        if (e == cudaSuccess) e = launch_b_resid(B->d_items, B->d_cta, B->grid, B->s);
        if (e == cudaSuccess) e = launch_b_reduce(B->d_items, count, nmax, 0, B->s);
        if (e == cudaSuccess) e = launch_b_trsv(B->d_items, count, 2, step, nmax, B->s);
        if (e == cudaSuccess) e = launch_b_init(B->d_items, count, step, 100, gam, rho, B->s);
        return e;
      });
      if (st < 0) return st;
    }
    st = capture(B, &G.iter, [&]() -> cudaError_t {
      cudaError_t e = launch_b_redeal(B->d_items, count, B->d_cta, B->grid, 0, B->s);
      if (e == cudaSuccess) e = launch_b_trsv(B->d_items, count, 0, 0, nmax, B->s);
      if (e == cudaSuccess) e = launch_b_inner(B->d_items, B->d_cta, B->grid, B->s);
      if (e == cudaSuccess) e = launch_b_reduce(B->d_items, count, nmax, 1, B->s);
      if (e == cudaSuccess) e = launch_b_trsv(B->d_items, count, 1, 0, nmax, B->s);
      if (e == cudaSuccess) e = launch_b_update(B->d_items, count, B->s);
      return e;
    });
    if (st < 0) return st;
    st = capture(B, &G.post, [&]() -> cudaError_t {
      return launch_b_trsv(B->d_items, count, 3, 0, nmax, B->s);
    });
    if (st < 0) return st;
  }
  // phase times (CUDA events on the batch's stream): pre (sketch, QR, setup),
  // step 0, step 1
  cudaEvent_t ev[4];
  for (auto &e : ev) BCU(cudaEventCreate(&e));
  int iters_run[2] = {0, 0};
  BCU(cudaEventRecord(ev[0], B->s));
  BCU(cudaGraphLaunch(G.pre, B->s));
  if (coop_qr) {
    B->qr_epoch = (B->qr_epoch >= (1 << 30)) ? 1 : B->qr_epoch + 1;
    BCU(launch_b_qr(B->d_items, B->d_qmap, B->qgrid, B->qr_epoch, kQrTimeoutNs, B->s));
  }
  BCU(cudaGraphLaunch(G.setup, B->s));
  BCU(cudaEventRecord(ev[1], B->s));
  {
    lsq_status st = read_states(B, count);
    if (st < 0) return st;
  }
  int q2max = 1;
  for (int i = 0; i < count; i++) q2max = std::max(q2max, B->h_st[i].q2);
  for (int step = 0; step < 2; step++) {
    BCU(cudaGraphLaunch(step == 0 ? G.step0 : G.step1, B->s));
    const int cap = step == 0 ? 100 : q2max;
    for (int it = 0; it < cap; it++) {
      BCU(cudaGraphLaunch(G.iter, B->s));
      iters_run[step]++;
      if (step == 0 && (it % kPollEvery) == kPollEvery - 1 && it + 1 < cap) {
        lsq_status st = read_states(B, count);
        if (st < 0) return st;
        bool all = true;
        for (int i = 0; i < count; i++) all = all && B->h_st[i].done;
        if (all) break;
      }
    }
    BCU(cudaGraphLaunch(G.post, B->s));
    BCU(cudaEventRecord(ev[2 + step], B->s));
    if (step == 0) {
      lsq_status st = read_states(B, count);
      if (st < 0) return st;
      for (int i = 0; i < count; i++) {
        if (infos) {
          std::memset(&infos[i], 0, sizeof(lsq_info));
          infos[i].iters[0] = B->h_st[i].iters;
          infos[i].resid0 = std::sqrt(B->h_st[i].r2);
          infos[i].thresh1 = B->h_st[i].thresh1;
        }
      }
    }
  }
  BCU(launch_b_copy_x(B->d_items, count, B->s));
  {
    lsq_status st = read_states(B, count);
    if (st < 0) return st;
  }
  float ms_pre = 0.f, ms_s0 = 0.f, ms_s1 = 0.f;
  cudaEventElapsedTime(&ms_pre, ev[0], ev[1]);
  cudaEventElapsedTime(&ms_s0, ev[1], ev[2]);
  cudaEventElapsedTime(&ms_s1, ev[2], ev[3]);
  for (auto &e : ev) cudaEventDestroy(e);
  lsq_status worst = LSQ_OK;
  for (int i = 0; i < count; i++) {
    const DevState &S = B->h_st[i];
    lsq_status st = LSQ_OK;
    if (S.nonfinite) st = LSQ_ERR_NONFINITE;
    else if (S.zero_col) st = LSQ_ERR_INVALID;
    else if (S.err) st = (lsq_status)S.err;
    else if (S.condest > 1.0 / (30.0 * kU)) st = LSQ_WARN_RANK_DEFICIENT;
    items[i].status = st;
    if (st < 0 && worst >= 0) worst = st;
    if (infos) {
      lsq_info &f = infos[i];
      f.iters[1] = S.iters;
      f.refine_steps = 2;
      f.path = LSQ_PREC_FP64;
      f.status = st;
      f.condest = S.condest;
      f.normest = S.normest;
      f.cnorm[0] = std::sqrt(S.cnorm2[0]);
      f.cnorm[1] = std::sqrt(S.cnorm2[1]);
      f.inner_kernel = 3;
      // the batch's phase times and the inner iterations it ran (lockstep:
      // the same for every item): sketch + QR + setup, step 1, step 2
      f.ms_sketch = ms_pre;
      f.ms_refine = ms_s0 + ms_s1;
      f.ms_total = ms_pre + ms_s0 + ms_s1;
      f.ms_inner_pass = ms_s1;
      f.ms_resid_pass = ms_s0;
      f.n_inner_pass = iters_run[0] + iters_run[1];
      f.n_resid_pass = iters_run[0];
      f.passes = 3 + f.iters[0] + f.iters[1];
      f.bytes_a = 8.0 * (double)items[i].m * (double)items[i].n * (double)(2 + f.passes);
    }
  }
  if (worst < 0) set_last_error("an item of the batch failed (see its status)");
  return worst;
}

// Host driver and C ABI (include/lsq.h) of the least-squares library.
//
// A solve is Alg. 1 of the paper with FOSSILS' Polyak (Alg. 2, Alg. 5) or
// SPIR's conjugate gradient (Alg. 3) as the inner solver and the practical
// rules of Sec. 4.2 / Alg. 4 (column scaling, d = 12n, zeta = 8,
// eta = sqrt(n/d), the step-1 stopping rule, the q0 count of Theorem 7.1 for
// step 2).  Every step is one of this library's kernels, enqueued on the
// plan's stream; the host only waits (a) once after the sketch and QR, for
// condest and the input checks, and (b) every few inner iterations of step 1
// to learn whether the device-side stop test has fired.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <vector>

#include "lsq_common.cuh"

using namespace lsq;

namespace {

thread_local std::string g_err;

lsq_status fail(lsq_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

#define LSQ_CU(call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(LSQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

#define LSQ_TRY(expr)                 \
  do {                                \
    lsq_status s_ = (expr);           \
    if (s_ < 0) return s_;            \
  } while (0)

constexpr uint64_t kBarrierTimeoutNs = 5ull * 1000 * 1000 * 1000;  // 5 s per inter-CTA wait
constexpr int kCondestIters = 10;
constexpr int kStopPollEvery = 4;  // step 1: read the device stop flag every 4 updates
constexpr int kHostChunksMax = 16;             // host entry: row chunks of A at most
constexpr double kHostChunkBytes = 128.0e6;    // and at least this many bytes each

}  // namespace

void lsq::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

struct lsq_plan_s {
  lsq_options o{};
  cudaStream_t s = nullptr;
  int dev = 0, nsm = 0;
  int64_t m = 0, n = 0, lda = 0;
  int d = 0, zeta = 0, npad = 0, gpass = 0, gqr = 0;
  int64_t m_cap = 0, n_cap = 0;      // sizes the workspace was allocated for
  int d_cap = 0, zeta_cap = 0;
  bool stepwise_qr = false;          // one launch per QR column (concurrent solves)
  uint64_t pat_key[4] = {0, 0, 0, 0};
  double eta = 0, alpha = 0, beta = 0;
  int32_t *pat_rows = nullptr;
  uint32_t *pat_sb = nullptr;
  bool pat_valid = false;
  // gather form of the sketch: source lists of the sketch rows (built with
  // the pattern), fixed-point scratch
  bool use_gather = false;
  int *tcnt = nullptr, *tlmax = nullptr, *colexp = nullptr, *cshift = nullptr;
  int64_t *tptr = nullptr;
  uint32_t *tsrc = nullptr;
  double *cpow = nullptr;
  long long *Qfix = nullptr, *Qbfix = nullptr;  // fixed-point copy of A and b (gather)
  double *SAb = nullptr, *W = nullptr, *part = nullptr, *r2part = nullptr, *cpart = nullptr;
  double *dcol = nullptr, *dinv = nullptr, *Rcm = nullptr, *Rrm = nullptr, *rinv = nullptr;
  double *Dt = nullptr;  // scaled diagonal blocks of R (launch_diag_tiles)
  double *t = nullptr, *vbuf = nullptr;
  double *xs = nullptr, *xo = nullptr, *c = nullptr, *g = nullptr, *dy = nullptr;
  double *dyold = nullptr, *z = nullptr, *h = nullptr, *w = nullptr, *res = nullptr, *p = nullptr;
  double *lsqr_s = nullptr;          // LSQR-SPIR: the m-vector of the bidiagonalisation
  // sketched Karlson-Walden estimate: [R; sqrt(lam) I] and its R factor
  double *W2 = nullptr, *R2cm = nullptr, *R2rm = nullptr, *rinv2 = nullptr, *Dt2 = nullptr;
  double *part2 = nullptr;           // compensated residual: (sum, error) partials
  double *vhead2 = nullptr, *xk = nullptr, *xko = nullptr, *gk = nullptr;
  int *qflag2 = nullptr;
  int qr2_epoch = 0;
  DevState *st = nullptr;
  DevState *st_host = nullptr;
  int *qflag = nullptr;              // QR: per-column "reflector published" flags
  int qr_epoch = 0;                  // value the flags take in the current QR launch
  cudaEvent_t ev[5] = {};
  // condest runs on a second stream, overlapping x0, the first residual and
  // c0 on the main one; the main stream joins it before the step-1 threshold
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  QrBlocked qb{};                    // blocked QR: T workspace, panel stream, events
  // CSR input of the solve in progress (lsq_solve_csr), else all NULL
  struct {
    const int64_t *rp = nullptr;
    const int32_t *col = nullptr;
    const double *val = nullptr;
    int64_t nnz = 0;
  } csr;
  bool condest_pending = false;
  double *stageA = nullptr, *stageb = nullptr, *stagex = nullptr;
  size_t stage_cap = 0;              // doubles of stageA
  // host entry: A copied in row chunks on a copy stream (one event per
  // chunk), the sketch of each chunk run as it lands (gather form only)
  cudaStream_t scopy = nullptr;
  cudaEvent_t ev_stage = nullptr;
  cudaEvent_t chunk_ev[kHostChunksMax] = {};
  int64_t chunk_row[kHostChunksMax + 1] = {};
  int host_chunks = 0;               // > 1: do_sketch waits per chunk
  bool sketched = false;
  bool use_eft = false;              // inner pass on the FP32 pipe
  bool want32 = false;               // the sketch pass writes the hi / lo planes of A
  bool planes_pending = false;       // the first residual pass of the solve writes them
  float *Ahi = nullptr, *Alo = nullptr;  // FP32 planes: hi = fl32(A), lo = A - hi
  int64_t ld32 = 0;
  bool use_df = false;               // inner pass in double-float on the planes
  int col_exp = 0;                   // all |A_ij| < 2^col_exp
  double *dcol_host = nullptr;
  // many right-hand sides (nrhs > 0)
  int k = 0;
  bool multi_planes = false;        // the planes hold the A of the last multi solve
  double *SBb = nullptr, *cpartB = nullptr, *mpart = nullptr, *mr2part = nullptr, *mT = nullptr;
  double *mpartdf = nullptr;  // partials of the batched double-float pass (k x gpass x npad)
  double *mXs = nullptr, *mXo = nullptr, *mC = nullptr, *mG = nullptr, *mDY = nullptr;
  double *mDYold = nullptr, *mZ = nullptr, *mH = nullptr, *mW = nullptr, *mstate = nullptr;
  int launches = 0;                 // kernels launched by the current call
  std::vector<cudaEvent_t> tev;     // timing: pass begin/end event pairs
  int tev_used = 0;
};

cudaError_t lsq::ensure_smem_attr(const void *fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int &have = done[{dev, fn}];
  if (have >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

namespace {

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  return cudaMalloc((void **)p, count * sizeof(T) + 16);
}

lsq_status validate(const lsq_options *o) {
  if (!o) return fail(LSQ_ERR_INVALID, "options is NULL");
  if (o->n < 1 || o->m < o->n) return fail(LSQ_ERR_INVALID, "need m >= n >= 1");
  if (o->n > LSQ_MAX_N) return fail(LSQ_ERR_INVALID, "n exceeds LSQ_MAX_N");
  if (o->lda != 0 && o->lda < o->n) return fail(LSQ_ERR_INVALID, "lda < n");
  const int64_t d = o->d ? o->d : 12 * o->n;
  if (d < o->n || d > (int64_t)1 << 24) return fail(LSQ_ERR_INVALID, "need n <= d <= 2^24");
  const int zeta = o->zeta ? o->zeta : 8;
  if (zeta < 1 || zeta > kMaxZeta || zeta > d) return fail(LSQ_ERR_INVALID, "need 1 <= zeta <= min(32, d)");
  if (o->max_inner < 0 || o->max_refine < 0 || o->max_refine > LSQ_MAX_REFINE)
    return fail(LSQ_ERR_INVALID, "max_inner / max_refine out of range");
  if (o->eta < 0 || o->eta >= 1) return fail(LSQ_ERR_INVALID, "eta must be in [0, 1)");
  if (o->precision < LSQ_PREC_AUTO || o->precision > LSQ_PREC_FP32_INNER)
    return fail(LSQ_ERR_INVALID, "unknown precision");
  if (o->qr_wait_us < 0) return fail(LSQ_ERR_INVALID, "qr_wait_us must be >= 0");
  if (o->kw_stop != 0 && o->kw_stop != 1) return fail(LSQ_ERR_INVALID, "kw_stop must be 0 or 1");
  if (o->nrhs < 0 || (o->nrhs > 0 && !multi_supported((int)o->n, o->nrhs)))
    return fail(LSQ_ERR_INVALID, "nrhs must be a multiple of 8 in [8, 64] with n <= 256");
  if (o->sparse != 0 && o->sparse != 1) return fail(LSQ_ERR_INVALID, "sparse must be 0 or 1");
  if (o->sparse && (o->nrhs != 0 || o->kw_stop != 0 || o->precision != LSQ_PREC_FP64))
    return fail(LSQ_ERR_INVALID, "a sparse plan needs precision FP64, nrhs = 0, kw_stop = 0");
  return LSQ_OK;
}

// Step-2 inner count: q0 of Theorem 7.1 with kappa -> condest and distortion
// 1.01 eta; Alg. 5 returns dy_(q) after q - 1 updates.
int step2_updates(double condest, double eta, int max_inner) {
  const double e = 1.01 * eta;
  double q0 = 11.0;
  if (e > 0.0 && std::isfinite(condest) && condest > 0.0) {
    const double v = 1.0 + 2.0 * std::log(1.0 / (condest * kU)) / std::log(1.0 / e);
    q0 = v > 11.0 ? v : 11.0;
  }
  int q = (int)std::ceil(q0) - 1;
  if (q < 1) q = 1;
  if (q > max_inner) q = max_inner;
  return q;
}

// Inner updates per refinement step of the FP32 tier: the q0 count of
// Theorem 7.1 with the FP32 unit roundoff 2^-24 in place of u (the inner
// solve only has to reach the accuracy its FP32 passes allow), at least 4.
int tier_updates(double condest, double eta, int max_inner) {
  const double u32 = 5.9604644775390625e-08;
  const double e = 1.01 * eta;
  double q0 = 4.0;
  if (e > 0.0 && std::isfinite(condest) && condest > 0.0) {
    const double v = 1.0 + 2.0 * std::log(1.0 / (condest * u32)) / std::log(1.0 / e);
    q0 = v > 4.0 ? v : 4.0;
  }
  int q = (int)std::ceil(q0) - 1;
  if (q < 1) q = 1;
  if (q > max_inner) q = max_inner;
  return q;
}

bool planes_ok(lsq_plan P);

// FP32 tier gate: the FP32 copy exists, the precision option asks for it (or
// AUTO and condest below the gate), and every column norm is in FP32 range.
bool tier_ok(lsq_plan P) {
  if (!P->want32) return false;
  const int prec = P->o.precision;
  if (prec == LSQ_PREC_FP64) return false;
  const double gate = P->o.fp32_cond_max > 0 ? P->o.fp32_cond_max : 1e5;
  if (prec == LSQ_PREC_AUTO && !(P->st_host->condest < gate)) return false;
  return planes_ok(P);
}

// Limit of each inter-CTA wait of the cooperative QR.
uint64_t qr_timeout_ns(lsq_plan P) {
  return P->o.qr_wait_us > 0 ? (uint64_t)P->o.qr_wait_us * 1000ull : kBarrierTimeoutNs;
}

// Flag value of the next QR launch: never 0 (the flags' initial value) and
// never the previous launch's.
int next_epoch(lsq_plan P) {
  P->qr_epoch = (P->qr_epoch >= (1 << 30)) ? 1 : P->qr_epoch + 1;
  return P->qr_epoch;
}

// The gather form of the sketch pays a one-off list build per pattern and
// wins on large problems; it needs row indices below 2^31.
constexpr double kGatherMinElems = 16777216.0;  // m n >= 2^24 (A >= 128 MB)
bool gather_size_ok(int64_t m, int64_t n) {
  return m < ((int64_t)1 << 31) && (double)m * (double)n >= kGatherMinElems;
}

// The sparse sign pattern of the current (m, d, zeta, seed), built once and
// cached, and for large problems the source lists of the gather sketch
// (the sketch falls back to the scatter form when a list is too long to
// sort in shared memory).
lsq_status ensure_pattern(lsq_plan P) {
  if (P->pat_valid) return LSQ_OK;
  LSQ_CU(launch_sketch_pattern(P->m, P->d, P->zeta, P->o.seed, P->pat_rows, P->pat_sb, P->s));
  P->launches++;
  P->use_gather = false;
  if (P->tsrc != nullptr && gather_size_ok(P->m, P->n)) {
    LSQ_CU(launch_sketch_lists(P->pat_rows, P->pat_sb, P->m, P->zeta, P->d, P->tcnt, P->tptr,
                               P->tsrc, P->tlmax, P->s));
    P->launches += 4;
    int lmax = 0;
    LSQ_CU(cudaMemcpyAsync(&lmax, P->tlmax, sizeof(int), cudaMemcpyDeviceToHost, P->s));
    LSQ_CU(cudaStreamSynchronize(P->s));
    P->use_gather = lmax <= sketch_list_max();
  }
  P->pat_valid = true;
  return LSQ_OK;
}

// Order the main stream after the condest launched by do_sketch.
lsq_status join_condest(lsq_plan P) {
  if (P->condest_pending) {
    LSQ_CU(cudaStreamWaitEvent(P->s, P->ev_join, 0));
    P->condest_pending = false;
  }
  return LSQ_OK;
}

lsq_status read_state(lsq_plan P) {
  LSQ_CU(cudaMemcpyAsync(P->st_host, P->st, sizeof(DevState), cudaMemcpyDeviceToHost, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  if (P->st_host->err != 0) return fail((lsq_status)P->st_host->err, "device-side wait timed out");
  return LSQ_OK;
}

// Timing events (opt-in): a growing pool of begin/end pairs.
cudaError_t tev_pair(lsq_plan P, int *idx) {
  while ((int)P->tev.size() < 2 * (P->tev_used + 1)) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    P->tev.push_back(e);
  }
  *idx = P->tev_used++;
  return cudaSuccess;
}

float tev_ms(lsq_plan P, int idx) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, P->tev[2 * idx], P->tev[2 * idx + 1]);
  return ms;
}

// The hi / lo planes hold every significant entry of A when each column
// norm is in [2^-40, 2^40] (entries below 2^-60 of their column's norm may
// lose their lo part, which is below 2^-84 of the column).
bool planes_ok(lsq_plan P) {
  for (int j = 0; j < (int)P->n; j++) {
    const double v = P->dcol_host[j];
    if (!(v >= std::ldexp(1.0, -40) && v <= std::ldexp(1.0, 40))) return false;
  }
  return true;
}

// The FP32-pipe inner pass needs every significant entry of A in FP32
// range after one common power-of-two scaling: all column norms within 2^20
// of the largest (column norms are the dcol of the column scaling).
void choose_inner_kernel(lsq_plan P) {
  P->use_eft = false;
  P->use_df = false;
  if (P->o.inner_fp64_fma || P->csr.rp != nullptr) return;
  if (P->want32 && planes_ok(P)) {
    P->use_df = true;
    return;
  }
  double mx = 0.0, mn = INFINITY;
  for (int j = 0; j < (int)P->n; j++) {
    const double v = P->dcol_host[j];
    if (!(v > 0.0) || !std::isfinite(v)) return;
    mx = v > mx ? v : mx;
    mn = v < mn ? v : mn;
  }
  int e = 0;
  std::frexp(mx, &e);  // mx < 2^e
  if (mn < std::ldexp(1.0, e - 20) || e > 100 || e < -100) return;
  P->col_exp = e;
  P->use_eft = true;
}

// defer_planes: on the gather path the prep pass leaves the hi / lo planes to
// the solve's first residual pass (planes_pending), which reads A anyway.
lsq_status do_sketch(lsq_plan P, const double *dA, const double *db, bool defer_planes) {
  if (!db || (!dA && P->csr.rp == nullptr)) return fail(LSQ_ERR_INVALID, "A or b is NULL");
  if (P->o.sparse && P->csr.rp == nullptr)
    return fail(LSQ_ERR_INVALID, "the plan was created for CSR input (lsq_solve_csr)");
  const int n = (int)P->n;
  P->launches = 0;
  P->tev_used = 0;
  LSQ_TRY(join_condest(P));  // a previous call that failed early may have left one running
  P->multi_planes = false;
  // fresh device state with alpha, beta
  std::memset(P->st_host, 0, sizeof(DevState));
  P->st_host->alpha = P->alpha;
  P->st_host->beta = P->beta;
  LSQ_CU(cudaMemcpyAsync(P->st, P->st_host, sizeof(DevState), cudaMemcpyHostToDevice, P->s));
  LSQ_CU(cudaEventRecord(P->ev[0], P->s));
  LSQ_TRY(ensure_pattern(P));
  int tk = -1;
  if (P->o.timing) {
    LSQ_CU(tev_pair(P, &tk));
    LSQ_CU(cudaEventRecord(P->tev[2 * tk], P->s));
  }
  const int nch = P->host_chunks;
  P->host_chunks = 0;
  P->planes_pending = false;
  if (P->csr.rp != nullptr) {
    // the structure and values first: a bad index must stop the solve before
    // any kernel indexes with it
    LSQ_CU(launch_csr_check(P->csr.rp, P->csr.col, P->csr.val, P->m, n, P->csr.nnz, db, P->st,
                            P->nsm, P->s));
    LSQ_TRY(read_state(P));
    if (P->st_host->err == LSQ_ERR_INVALID)
      return fail(LSQ_ERR_INVALID, "not a CSR matrix of m x n with nnz entries");
    if (P->st_host->nonfinite) return fail(LSQ_ERR_NONFINITE, "A or b holds NaN or Inf");
    LSQ_CU(cudaMemsetAsync(P->SAb, 0, sizeof(double) * (size_t)P->d * (n + 1), P->s));
    LSQ_CU(launch_csr_sketch(P->csr.rp, P->csr.col, P->csr.val, P->m, n, db, P->d, P->zeta,
                             P->pat_rows, P->pat_sb, P->SAb, P->cpart, P->gpass, P->npad, P->s));
    P->launches += 2;
  } else if (P->use_gather) {
    const bool planes = P->want32 && !defer_planes;
    P->planes_pending = P->want32 && defer_planes;
    // one chunk, or the host entry's row chunks as their copies complete
    for (int c = 0; c < std::max(nch, 1); c++) {
      const int64_t r0 = nch > 1 ? P->chunk_row[c] : 0, r1 = nch > 1 ? P->chunk_row[c + 1] : P->m;
      if (nch > 1) LSQ_CU(cudaStreamWaitEvent(P->s, P->chunk_ev[c], 0));
      LSQ_CU(launch_sketch_prep(dA + r0 * P->lda, P->lda, r1 - r0, n, db + r0, P->cpart, P->gpass,
                                P->npad, P->colexp, planes ? P->Ahi + r0 * P->ld32 : nullptr,
                                planes ? P->Alo + r0 * P->ld32 : nullptr, P->ld32, P->s, c > 0));
      LSQ_CU(launch_sketch_gather(dA, P->lda, n, db, P->d, P->npad, P->tptr, P->tsrc, P->colexp,
                                  P->tlmax, P->cshift, P->cpow, P->SAb, P->st, P->s, r0, r1,
                                  c > 0, P->Qfix, P->Qbfix, (n + 1) & ~1, P->gpass));
      P->launches += 4;  // prep, fixed parameters, fixed-point copy, gather
    }
    P->launches -= 1;  // counted below with the finalize
  } else {
    for (int c = 0; c < nch; c++) LSQ_CU(cudaStreamWaitEvent(P->s, P->chunk_ev[c], 0));
    LSQ_CU(cudaMemsetAsync(P->SAb, 0, sizeof(double) * (size_t)P->d * (n + 1), P->s));
    LSQ_CU(launch_sketch(dA, P->lda, P->m, n, db, P->d, P->zeta, P->pat_rows, P->pat_sb, P->SAb,
                         P->cpart, P->gpass, P->npad, P->want32 ? P->Ahi : nullptr,
                         P->want32 ? P->Alo : nullptr, P->ld32, P->s));
  }
  if (tk >= 0) LSQ_CU(cudaEventRecord(P->tev[2 * tk + 1], P->s));
  LSQ_CU(launch_sketch_finalize(P->cpart, P->gpass, P->npad, n, P->d, P->zeta, P->o.col_scale,
                                P->SAb, P->W, P->dcol, P->dinv, P->st, P->s));
  LSQ_CU(cudaEventRecord(P->ev[1], P->s));
  P->launches += 3 + 5;  // sketch, colnorm, transpose; qr, extract, tiles, condest, x0 solve
  if (P->stepwise_qr)
    LSQ_CU(launch_qr_stepwise(P->W, P->d, n, n + 1, P->vbuf, qr_step_grid(n + 1, P->nsm), P->s));
  else
    LSQ_CU(launch_qr(P->W, P->d, n, n + 1, P->vbuf, P->qflag, next_epoch(P), P->st,
                     qr_grid(n + 1, P->nsm), qr_timeout_ns(P), P->s, &P->qb));
  LSQ_CU(launch_extract_r(P->W, P->d, n, 1, P->Rcm, P->Rrm, P->rinv, P->t, P->s));
  LSQ_CU(launch_diag_tiles(P->Rcm, P->Rrm, P->rinv, n, P->Dt, P->s));
  LSQ_CU(cudaEventRecord(P->ev_fork, P->s));
  LSQ_CU(cudaStreamWaitEvent(P->s2, P->ev_fork, 0));
  LSQ_CU(launch_condest(P->Rcm, P->Rrm, P->rinv, P->Dt, n, kCondestIters, P->st, P->s2));
  LSQ_CU(cudaEventRecord(P->ev_join, P->s2));
  P->condest_pending = true;
  // sketch-and-solve x0 = R^{-1} t (scaled coordinates) and x0 / d (original)
  LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->t, nullptr, P->xs, P->dinv, P->xo,
                     nullptr, &P->st->x0norm2, nullptr, P->s, 1, 0,
                       &P->st->err));
  LSQ_CU(cudaEventRecord(P->ev[2], P->s));
  LSQ_CU(cudaMemcpyAsync(P->dcol_host, P->dcol, sizeof(double) * n, cudaMemcpyDeviceToHost, P->s));
  LSQ_TRY(read_state(P));
  choose_inner_kernel(P);
  if (P->st_host->nonfinite) return fail(LSQ_ERR_NONFINITE, "A or b holds NaN or Inf");
  if (P->st_host->zero_col) return fail(LSQ_ERR_INVALID, "A has a zero column (column scaling)");
  P->sketched = true;
  return LSQ_OK;
}

// Enqueue the sketched Karlson-Walden estimate (eq. (sketched-kw)) of the
// iterate xs (scaled coordinates) / xo (= D^-1 xs, original) into
// st->kw_est: one compensated (Dot2) FP64 residual pass, on the scaled
// problem (r = b - fl(A D^-1) xs, g = fl(A D^-1)^T r) when `scaled`, else on
// the original one (r = b - A xo, g = D^-1 A^T r), ||r||^2, the stacked matrix [R; sqrt(lam) I], its Householder QR (the cooperative QR
// kernel, d = 2n), the triangular solve R_lam^T y = g and the prefactor.
// st->bnorm2 must hold ||b||^2.
lsq_status kw_eval(lsq_plan P, const double *dA, const double *db, const double *xs,
                   const double *xo, bool scaled) {
  const int n = (int)P->n;
  if (scaled) {
    // the scaled problem fl(A D^-1) with the scaled iterate xs
    LSQ_CU(launch_pass_resid_dot2(dA, P->lda, P->m, n, db, xs, P->dinv, P->part2, P->r2part,
                                  P->gpass, P->npad, P->s));
    LSQ_CU(launch_reduce_dot2(P->part2, P->gpass, P->npad, n, nullptr, P->gk, P->r2part,
                              &P->st->kw_r2, P->s));
  } else {
    // A and the caller's xo; g = D^-1 A^T r
    LSQ_CU(launch_pass_resid_dot2(dA, P->lda, P->m, n, db, xo, nullptr, P->part2, P->r2part,
                                  P->gpass, P->npad, P->s));
    LSQ_CU(launch_reduce_dot2(P->part2, P->gpass, P->npad, n, P->dinv, P->gk, P->r2part,
                              &P->st->kw_r2, P->s));
  }
  LSQ_CU(launch_kw_build(P->Rcm, n, P->dcol, P->dinv, xs, P->W2, P->st, P->s));
  P->qr2_epoch = (P->qr2_epoch >= (1 << 30)) ? 1 : P->qr2_epoch + 1;
  LSQ_CU(launch_qr(P->W2, 2 * n, n, n, P->vhead2, P->qflag2, P->qr2_epoch, P->st,
                   qr_grid(n, P->nsm), qr_timeout_ns(P), P->s, &P->qb));
  LSQ_CU(launch_extract_r(P->W2, 2 * n, n, 0, P->R2cm, P->R2rm, P->rinv2, nullptr, P->s));
  LSQ_CU(launch_diag_tiles(P->R2cm, P->R2rm, P->rinv2, n, P->Dt2, P->s));
  LSQ_CU(launch_trsv(P->R2cm, P->R2rm, P->rinv2, P->Dt2, n, 1, P->gk, nullptr, P->gk, nullptr,
                     nullptr, nullptr, &P->st->kw_y2, nullptr, P->s, 1, 0, &P->st->err));
  LSQ_CU(launch_kw_finish(P->st, P->s));
  P->launches += 9;
  return LSQ_OK;
}

// ||A D^-1||_F from the column norms (sqrt(n) with column scaling).
double scaled_fro(lsq_plan P) {
  double s = 0.0;
  for (int j = 0; j < (int)P->n; j++) {
    const double c = P->o.col_scale ? 1.0 : P->dcol_host[j];
    s += c * c;
  }
  return std::sqrt(s);
}

lsq_status run_solve(lsq_plan P, int method, const double *dA, const double *db, double *dx,
                     lsq_info *info) {
  if (!dx) return fail(LSQ_ERR_INVALID, "x is NULL");
  const int n = (int)P->n;
  LSQ_TRY(do_sketch(P, dA, db, true));
  const int max_inner = P->o.max_inner ? P->o.max_inner : 100;
  const int nref = P->o.max_refine ? P->o.max_refine : 2;
  const double gam = P->o.stop_gamma, rho = P->o.stop_rho;
  // the FP32 tier is chosen on condest up front; the FP64 path needs it only
  // for the step-1 threshold (device) and the step-2 count (host, later)
  if (P->o.precision == LSQ_PREC_AUTO || P->o.precision == LSQ_PREC_FP32_INNER) {
    LSQ_TRY(join_condest(P));
    LSQ_TRY(read_state(P));
  }
  // method 2 (LSQR-based SPIR) keeps its passes on A's FP64-class forms
  const bool tier = method != 2 && tier_ok(P);
  const int q32 = tier ? tier_updates(P->st_host->condest, P->eta, max_inner) : 0;
  int q2 = -1;  // set from condest once step 1 has read the device state
  const int nsteps_max = tier ? std::min(LSQ_MAX_REFINE, std::max(nref, 6)) : nref;
  // bytes of A per pass: 8 m n dense; 12 nnz + 8 (m + 1) for CSR
  const double mn8 = P->csr.rp ? 12.0 * (double)P->csr.nnz + 8.0 * (double)(P->m + 1)
                               : 8.0 * (double)P->m * (double)n;
  double bytes_a = mn8 + (P->want32 ? mn8 : 0.0);  // sketch pass (+ hi / lo planes)
  int passes = 1;
  int iters[LSQ_MAX_REFINE] = {0};
  double resid0 = 0.0, cprev = INFINITY, kw_last = 0.0;
  int nsteps = 0;
  std::vector<int> resid_ev, inner_ev[LSQ_MAX_REFINE];
  for (int i = 0; i < nsteps_max; i++) {
    int tk = -1;
    if (P->o.timing) {
      LSQ_CU(tev_pair(P, &tk));
      resid_ev.push_back(tk);
      LSQ_CU(cudaEventRecord(P->tev[2 * tk], P->s));
    }
    const bool planes = P->planes_pending;
    P->planes_pending = false;
    if (P->csr.rp)
      LSQ_CU(launch_csr_pass(1, P->csr.rp, P->csr.col, P->csr.val, P->m, db, P->xo, P->part,
                             P->r2part, P->gpass, P->npad, nullptr, nullptr,
                             method == 2 ? P->lsqr_s : nullptr, P->s));
    else
      LSQ_CU(launch_pass_resid(dA, P->lda, P->m, n, db, P->xo, P->part, P->r2part, P->gpass,
                               P->npad, P->s, planes ? P->Ahi : nullptr,
                               planes ? P->Alo : nullptr, P->ld32, nullptr, nullptr,
                               method == 2 ? P->lsqr_s : nullptr));
    if (tk >= 0) LSQ_CU(cudaEventRecord(P->tev[2 * tk + 1], P->s));
    P->launches += 3 + (i == 0 ? 1 : 0) + 1;  // resid, reduce, trsv, [thresh], init
    LSQ_CU(launch_reduce(P->part, P->gpass, P->npad, n, P->dinv, P->g, P->r2part, &P->st->r2,
                         nullptr, P->s));
    passes++;
    LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 1, P->g, nullptr, P->c, nullptr, nullptr,
                       nullptr, &P->st->cnorm2[i], nullptr, P->s, 1, 0,
                       &P->st->err));
    if (i == 0) {
      LSQ_TRY(join_condest(P));
      LSQ_CU(launch_set_thresh(gam, rho, P->st, P->s));
    }
    if (i == 1 && q2 < 0) q2 = step2_updates(P->st_host->condest, P->eta, max_inner);
    bytes_a += mn8;
    if (tier) {
      // refine until ||c_i|| stops halving (the FP64 residual's noise floor)
      LSQ_TRY(read_state(P));
      const double cn = std::sqrt(P->st_host->cnorm2[i]);
      if (i == 0) resid0 = std::sqrt(P->st_host->r2);
      if ((i >= 2 && !(cn <= 0.5 * cprev)) || cn == 0.0) break;
      cprev = cn;
    }
    const bool fixed = P->o.fixed_inner > 0;
    // Alg. 4's step-2 test (kw_stop): up to max_inner updates, the sketched KW
    // estimate checked after updates 1, 6, 11, ... (reading: the inner index)
    const bool kw = P->o.kw_stop && i == 1 && !fixed && !tier;
    const int cap = fixed ? P->o.fixed_inner : tier ? q32 : (i == 0 || kw) ? max_inner : q2;
    const int use_thresh = (!fixed && !tier && i == 0) ? 1 : 0;
    if (kw) LSQ_CU(launch_bnorm2(db, P->m, P->st, P->s));
    if (method == 2)
      LSQ_CU(launch_lsqr_init(n, P->c, i, P->p, P->res, P->dy, cap, use_thresh, P->st, P->s));
    else
      LSQ_CU(launch_inner_init(method, n, P->c, P->dy, P->dyold, P->res, P->p, cap, use_thresh,
                               P->st, P->s));
    // Under the step-2 test the inner passes are strict FP64: the double-float
    // pass's operator holds A to 2^-48, which leaves step 2's answer a few u
    // ||A||_F from backward stable on kappa ~ 1e12 problems, above the bound.
    const bool df = P->use_df && !kw, eft = P->use_eft && !kw;
    for (int it = 0; it < cap; it++) {
      const double *src = (method == 0) ? P->dy : P->p;
      // z = D^{-1} R^{-1} src;  h = D^{-1} A^T (A z);  w = R^{-T} h
      LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, src, nullptr, nullptr, P->dinv, P->z,
                         nullptr, nullptr, P->st, P->s, 1, 0,
                       &P->st->err));
      int tj = -1;
      if (P->o.timing) {
        LSQ_CU(tev_pair(P, &tj));
        inner_ev[i].push_back(tj);
        LSQ_CU(cudaEventRecord(P->tev[2 * tj], P->s));
      }
      if (P->csr.rp)
        LSQ_CU(launch_csr_pass(method == 2 ? 1 : 0, P->csr.rp, P->csr.col, P->csr.val, P->m,
                               method == 2 ? P->lsqr_s : nullptr, P->z, P->part, P->r2part,
                               P->gpass, P->npad, P->st,
                               method == 2 ? &P->st->lq_bscale : nullptr,
                               method == 2 ? P->lsqr_s : nullptr, P->s));
      else if (method == 2 && df)
        LSQ_CU(launch_pass_lsqr_df(P->Ahi, P->Alo, P->ld32, P->m, n, P->z, P->lsqr_s,
                                   &P->st->lq_bscale, P->part, P->r2part, P->gpass, P->npad, P->st,
                                   &P->st->err, P->s));
      else if (method == 2)
        LSQ_CU(launch_pass_resid(dA, P->lda, P->m, n, P->lsqr_s, P->z, P->part, P->r2part,
                                 P->gpass, P->npad, P->s, nullptr, nullptr, 0, P->st,
                                 &P->st->lq_bscale, P->lsqr_s));
      else if (tier)
        LSQ_CU(launch_pass_atax32(P->Ahi, P->ld32, P->m, n, P->z, P->part, P->gpass, P->npad,
                                  P->st, &P->st->err, P->s));
      else if (df)
        LSQ_CU(launch_pass_atax_df(P->Ahi, P->Alo, P->ld32, P->m, n, P->z, P->part, P->gpass,
                                   P->npad, P->st, &P->st->err, P->s));
      else if (eft)
        LSQ_CU(launch_pass_atax_eft(dA, P->lda, P->m, n, P->z, P->col_exp, P->part, P->gpass,
                                    P->npad, P->st, P->s));
      else
        LSQ_CU(launch_pass_atax(dA, P->lda, P->m, n, P->z, P->part, P->gpass, P->npad, P->st,
                                P->s));
      if (tj >= 0) LSQ_CU(cudaEventRecord(P->tev[2 * tj + 1], P->s));
      P->launches += 5;
      LSQ_CU(launch_reduce(P->part, P->gpass, P->npad, n, P->dinv, P->h,
                           method == 2 ? P->r2part : nullptr,
                           method == 2 ? &P->st->lq_b2 : nullptr, P->st, P->s));
      LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 1, P->h, nullptr, P->w, nullptr, nullptr,
                         nullptr, nullptr, P->st, P->s, 1, 0,
                       &P->st->err));
      if (method == 0)
        LSQ_CU(launch_polyak_update(n, P->c, P->w, P->dy, P->dyold, P->st, P->s));
      else if (method == 1)
        LSQ_CU(launch_cg_update(n, P->w, P->p, P->res, P->dy, P->st, P->s));
      else
        LSQ_CU(launch_lsqr_update(n, P->w, P->p, P->res, P->dy, P->st, P->s));
      if (use_thresh && (it % kStopPollEvery) == kStopPollEvery - 1 && it + 1 < cap) {
        LSQ_TRY(read_state(P));
        if (P->st_host->done) break;
      }
      if (kw && it % 5 == 0) {
        // x_hat = x_s + R^{-1} dy (scaled) and D^{-1} x_hat, then the estimate
        LSQ_CU(cudaMemcpyAsync(P->xk, P->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->s));
        LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->dy, nullptr, nullptr, P->dinv,
                           P->xko, P->xk, nullptr, nullptr, P->s, 1, 0, &P->st->err));
        LSQ_TRY(kw_eval(P, dA, db, P->xk, P->xko, true));
        LSQ_TRY(read_state(P));
        kw_last = P->st_host->kw_est;
        if (P->st_host->done || kw_last < kUKwStop * scaled_fro(P)) break;
      }
    }
    // x_s += R^{-1} dy ; x_o = D^{-1} x_s
    LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->dy, nullptr, nullptr, P->dinv, P->xo,
                       P->xs, nullptr, nullptr, P->s, 1, 0,
                       &P->st->err));
    P->launches++;
    LSQ_TRY(read_state(P));
    iters[i] = P->st_host->iters;
    if (i == 0 && !tier) resid0 = std::sqrt(P->st_host->r2);
    passes += iters[i];
    bytes_a += (tier ? mn8 / 2 : mn8) * iters[i];
    nsteps = i + 1;
  }
  LSQ_CU(cudaMemcpyAsync(dx, P->xo, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaEventRecord(P->ev[3], P->s));
  LSQ_TRY(read_state(P));
  const DevState &S = *P->st_host;
  lsq_status status = LSQ_OK;
  if (S.condest > 1.0 / (30.0 * kU)) status = LSQ_WARN_RANK_DEFICIENT;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int i = 0; i < nsteps; i++) {
      info->iters[i] = iters[i];
      info->cnorm[i] = std::sqrt(S.cnorm2[i]);
    }
    info->refine_steps = nsteps;
    info->path = tier ? LSQ_PREC_FP32_INNER : LSQ_PREC_FP64;
    info->bytes_a = bytes_a;
    info->passes = passes;
    info->status = status;
    info->condest = S.condest;
    info->normest = S.normest;
    info->thresh1 = S.thresh1;
    float ms = 0;
    cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]);
    info->ms_sketch = ms;
    cudaEventElapsedTime(&ms, P->ev[1], P->ev[2]);
    info->ms_qr = ms;
    cudaEventElapsedTime(&ms, P->ev[2], P->ev[3]);
    info->ms_refine = ms;
    cudaEventElapsedTime(&ms, P->ev[0], P->ev[3]);
    info->ms_total = ms;
    info->launches = P->launches;
    info->inner_kernel = tier ? 2 : P->use_df ? 3 : (P->use_eft && method != 2) ? 1 : 0;
    if (P->o.timing) {
      for (int k : resid_ev) {
        info->ms_resid_pass += tev_ms(P, k);
        info->n_resid_pass++;
      }
      // only the launches before the stop decision did work
      for (int i = 0; i < nsteps; i++)
        for (int j = 0; j < (int)inner_ev[i].size() && j < iters[i]; j++) {
          info->ms_inner_pass += tev_ms(P, inner_ev[i][j]);
          info->n_inner_pass++;
        }
      info->ms_sketch_pass = tev_ms(P, 0);
    }
  }
  if (info) {
    info->resid0 = resid0;
    info->be_sketch_est = kw_last;
  }
  return status;
}

// Many right-hand sides, inner pass in double-float on the planes: the
// k-tiled pass (every row block of A applied to all k vectors while it is in
// shared memory) when its tiles fit, else one launch of the single-vector
// pass over k grid rows (each vector re-reads A).  H (n x k column-major) =
// scale .* A^T (A Z).
cudaError_t launch_multi_df_pass(lsq_plan P, const double *Z, double *H, const double *scale,
                                 const DevState *gate) {
  const int n = (int)P->n, k = P->k;
  if (multi_df_supported(n, k, P->ld32)) {
    cudaError_t e = launch_pass_atax_df_multi(P->Ahi, P->Alo, P->ld32, P->m, n, Z, k, P->mpartdf,
                                              P->nsm, P->npad, gate, &P->st->err, P->s);
    if (e != cudaSuccess) return e;
    return launch_reduce_batched(P->mpartdf, P->nsm, P->npad, n, k, scale, H, gate, P->s);
  }
  const int64_t pstride = (int64_t)P->gpass * P->npad;
  cudaError_t e = launch_pass_atax_df(P->Ahi, P->Alo, P->ld32, P->m, n, Z, P->mpartdf, P->gpass,
                                      P->npad, gate, &P->st->err, P->s, k, n, pstride);
  if (e != cudaSuccess) return e;
  return launch_reduce_batched(P->mpartdf, P->gpass, P->npad, n, k, scale, H, gate, P->s);
}

// FOSSILS for k right-hand sides sharing one sketch and one QR.
lsq_status run_solve_multi(lsq_plan P, const double *dA, const double *dB, int64_t ldb,
                           double *dX, lsq_info *info) {
  if (P->k <= 0) return fail(LSQ_ERR_INVALID, "plan was created with nrhs = 0");
  if (!dA || !dB || !dX) return fail(LSQ_ERR_INVALID, "NULL argument");
  const int n = (int)P->n, k = P->k, d = P->d;
  if (ldb == 0) ldb = k;
  if (ldb < k) return fail(LSQ_ERR_INVALID, "ldb < nrhs");
  P->launches = 0;
  P->tev_used = 0;
  double *dn2 = P->mstate, *thr = P->mstate + k, *x0n2 = P->mstate + 2 * k;
  double *r2 = P->mstate + 3 * k, *cn2 = P->mstate + 4 * k;
  std::memset(P->st_host, 0, sizeof(DevState));
  P->st_host->alpha = P->alpha;
  P->st_host->beta = P->beta;
  LSQ_CU(cudaMemcpyAsync(P->st, P->st_host, sizeof(DevState), cudaMemcpyHostToDevice, P->s));
  LSQ_CU(cudaEventRecord(P->ev[0], P->s));
  LSQ_TRY(ensure_pattern(P));
  // one sketch S for [A B]: A's columns (with their norms), then B's
  LSQ_CU(cudaMemsetAsync(P->SAb, 0, sizeof(double) * (size_t)d * (n + 1), P->s));
  LSQ_CU(cudaMemsetAsync(P->SBb, 0, sizeof(double) * (size_t)d * (k + 1), P->s));
  LSQ_CU(launch_sketch(dA, P->lda, P->m, n, nullptr, d, P->zeta, P->pat_rows, P->pat_sb, P->SAb,
                       P->cpart, P->gpass, P->npad, P->want32 ? P->Ahi : nullptr,
                       P->want32 ? P->Alo : nullptr, P->ld32, P->s));
  LSQ_CU(launch_sketch(dB, ldb, P->m, k, nullptr, d, P->zeta, P->pat_rows, P->pat_sb, P->SBb,
                       P->cpartB, P->gpass, pass_npad(k), nullptr, nullptr, 0, P->s));
  LSQ_CU(launch_sketch_finalize(P->cpart, P->gpass, P->npad, n, d, P->zeta, P->o.col_scale,
                                P->SAb, P->W, P->dcol, P->dinv, P->st, P->s));
  LSQ_CU(launch_sketch_b_to_w(P->SBb, d, n, k, P->zeta, P->W, P->st, P->s));
  LSQ_CU(cudaEventRecord(P->ev[1], P->s));
  LSQ_CU(launch_qr(P->W, d, n, n + k, P->vbuf, P->qflag, next_epoch(P), P->st,
                   qr_grid(n + k, P->nsm), qr_timeout_ns(P), P->s, &P->qb));
  LSQ_CU(launch_extract_r(P->W, d, n, k, P->Rcm, P->Rrm, P->rinv, P->mT, P->s));
  LSQ_CU(launch_diag_tiles(P->Rcm, P->Rrm, P->rinv, n, P->Dt, P->s));
  LSQ_CU(launch_condest(P->Rcm, P->Rrm, P->rinv, P->Dt, n, kCondestIters, P->st, P->s));
  LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->mT, nullptr, P->mXs, P->dinv, P->mXo,
                     nullptr, x0n2, nullptr, P->s, k, n));
  LSQ_CU(cudaEventRecord(P->ev[2], P->s));
  P->launches += 12;
  LSQ_CU(cudaMemcpyAsync(P->dcol_host, P->dcol, sizeof(double) * n, cudaMemcpyDeviceToHost, P->s));
  LSQ_TRY(read_state(P));
  // the inner pass: all k vectors through the double-float pass on the planes
  // (one batched launch) unless the planes are off or out of range, else the
  // FP64 tensor-core contraction
  choose_inner_kernel(P);
  const bool multi_df = P->use_df;
  P->multi_planes = P->want32;  // the sketch above wrote the planes of this A
  if (P->st_host->nonfinite) return fail(LSQ_ERR_NONFINITE, "A or B holds NaN or Inf");
  if (P->st_host->zero_col) return fail(LSQ_ERR_INVALID, "A has a zero column (column scaling)");
  const int max_inner = P->o.max_inner ? P->o.max_inner : 100;
  const int nref = P->o.max_refine ? P->o.max_refine : 2;
  const int q2 = step2_updates(P->st_host->condest, P->eta, max_inner);
  int iters[LSQ_MAX_REFINE] = {0};
  double cmax[LSQ_MAX_REFINE] = {0};
  std::vector<double> hc(k);
  std::vector<int> inner_ev[LSQ_MAX_REFINE];
  for (int i = 0; i < nref; i++) {
    LSQ_CU(launch_multi_resid(dA, P->lda, P->m, n, k, dB, ldb, P->mXo, P->mpart, P->mr2part,
                              P->nsm, P->s));
    LSQ_CU(launch_multi_reduce(P->mpart, P->nsm, n, k, P->dinv, P->mG, P->mr2part, r2, nullptr,
                               P->s));
    LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 1, P->mG, nullptr, P->mC, nullptr, nullptr,
                       nullptr, cn2, nullptr, P->s, k, n));
    if (i == 0)
      LSQ_CU(launch_multi_thresh(k, P->o.stop_gamma, P->o.stop_rho, x0n2, r2, thr, P->st, P->s));
    const bool fixed = P->o.fixed_inner > 0;
    const int cap = fixed ? P->o.fixed_inner : (i == 0 ? max_inner : q2);
    const int use_thresh = (!fixed && i == 0) ? 1 : 0;
    LSQ_CU(launch_multi_init(n, k, P->mC, P->mDY, P->mDYold, cap, use_thresh, P->st, P->s));
    P->launches += 5;
    for (int it = 0; it < cap; it++) {
      LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->mDY, nullptr, nullptr, P->dinv, P->mZ,
                         nullptr, nullptr, P->st, P->s, k, n));
      int tj = -1;
      if (P->o.timing) {
        LSQ_CU(tev_pair(P, &tj));
        inner_ev[i].push_back(tj);
        LSQ_CU(cudaEventRecord(P->tev[2 * tj], P->s));
      }
      if (multi_df) {
        LSQ_CU(launch_multi_df_pass(P, P->mZ, P->mH, P->dinv, P->st));
        if (tj >= 0) LSQ_CU(cudaEventRecord(P->tev[2 * tj + 1], P->s));
      } else {
        LSQ_CU(launch_multi_atax(dA, P->lda, P->m, n, k, P->mZ, P->mpart, P->nsm, P->st, P->s));
        if (tj >= 0) LSQ_CU(cudaEventRecord(P->tev[2 * tj + 1], P->s));
        LSQ_CU(launch_multi_reduce(P->mpart, P->nsm, n, k, P->dinv, P->mH, nullptr, nullptr,
                                   P->st, P->s));
      }
      LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 1, P->mH, nullptr, P->mW, nullptr, nullptr,
                         nullptr, nullptr, P->st, P->s, k, n));
      LSQ_CU(launch_multi_polyak(n, k, P->mC, P->mW, P->mDY, P->mDYold, dn2, thr, P->st, P->s));
      P->launches += 6;
      if (use_thresh && (it % kStopPollEvery) == kStopPollEvery - 1 && it + 1 < cap) {
        LSQ_TRY(read_state(P));
        if (P->st_host->done) break;
      }
    }
    LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, n, 0, P->mDY, nullptr, nullptr, P->dinv, P->mXo,
                       P->mXs, nullptr, nullptr, P->s, k, n));
    P->launches++;
    LSQ_CU(cudaMemcpyAsync(hc.data(), cn2, sizeof(double) * k, cudaMemcpyDeviceToHost, P->s));
    LSQ_TRY(read_state(P));
    iters[i] = P->st_host->iters;
    for (int c = 0; c < k; c++) cmax[i] = std::max(cmax[i], std::sqrt(hc[c]));
  }
  LSQ_CU(launch_cm_to_rm(P->mXo, n, k, dX, P->s));
  LSQ_CU(cudaEventRecord(P->ev[3], P->s));
  P->launches++;
  LSQ_TRY(read_state(P));
  const DevState &S = *P->st_host;
  lsq_status status = (S.condest > 1.0 / (30.0 * kU)) ? LSQ_WARN_RANK_DEFICIENT : LSQ_OK;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    for (int i = 0; i < nref; i++) {
      info->iters[i] = iters[i];
      info->cnorm[i] = cmax[i];
    }
    info->refine_steps = nref;
    info->path = LSQ_PREC_FP64;
    info->inner_kernel = !multi_df ? 4 : multi_df_supported(n, k, P->ld32) ? 5 : 3;
    info->passes = 2 + nref + iters[0] + iters[1];
    info->status = status;
    info->condest = S.condest;
    info->normest = S.normest;
    info->launches = P->launches;
    info->bytes_a = 8.0 * (double)P->m * n * (1 + nref + iters[0] + (nref > 1 ? iters[1] : 0));
    float ms = 0;
    cudaEventElapsedTime(&ms, P->ev[0], P->ev[1]);
    info->ms_sketch = ms;
    cudaEventElapsedTime(&ms, P->ev[1], P->ev[2]);
    info->ms_qr = ms;
    cudaEventElapsedTime(&ms, P->ev[2], P->ev[3]);
    info->ms_refine = ms;
    cudaEventElapsedTime(&ms, P->ev[0], P->ev[3]);
    info->ms_total = ms;
    if (P->o.timing)
      for (int i = 0; i < nref; i++)
        for (int j = 0; j < (int)inner_ev[i].size() && j < iters[i]; j++) {
          info->ms_inner_pass += tev_ms(P, inner_ev[i][j]);
          info->n_inner_pass++;
        }
  }
  P->sketched = false;  // the plan's single-RHS R / x0 no longer describe one problem
  return status;
}

// Derived per-problem fields of a plan (sizes within capacity, Polyak
// coefficients, pass padding); invalidates the cached sketch pattern when its
// key (m, d, zeta, seed) changes.
void configure_fields(lsq_plan P, const lsq_options *opt) {
  P->o = *opt;
  P->m = opt->m;
  P->n = opt->n;
  P->lda = opt->lda ? opt->lda : opt->n;
  P->d = opt->d ? opt->d : (int)(12 * opt->n);
  P->zeta = opt->zeta ? opt->zeta : 8;
  P->eta = opt->eta > 0 ? opt->eta : std::sqrt((double)P->n / (double)P->d);
  P->beta = P->eta * P->eta;
  P->alpha = (1.0 - P->beta) * (1.0 - P->beta);
  if (P->o.max_inner == 0) P->o.max_inner = 100;
  if (P->o.max_refine == 0) P->o.max_refine = 2;
  P->npad = pass_npad((int)P->n);
  P->ld32 = (P->n + 3) / 4 * 4;
  P->want32 = (P->Ahi != nullptr) &&
              (!opt->inner_fp64_fma || opt->precision == LSQ_PREC_AUTO ||
               opt->precision == LSQ_PREC_FP32_INNER);
  const uint64_t key[4] = {(uint64_t)P->m, (uint64_t)P->d, (uint64_t)P->zeta, opt->seed};
  if (std::memcmp(key, P->pat_key, sizeof(key)) != 0) {
    std::memcpy(P->pat_key, key, sizeof(key));
    P->pat_valid = false;
  }
  P->sketched = false;
  P->multi_planes = false;
}

void free_plan(lsq_plan P) {
  if (!P) return;
  void *bufs[] = {P->pat_rows, P->pat_sb, P->SAb, P->W, P->part, P->r2part, P->cpart, P->dcol, P->dinv,
                  P->Rcm, P->Rrm, P->rinv, P->Dt, P->t, P->vbuf, P->xs, P->xo, P->c, P->g, P->dy,
                  P->dyold, P->z, P->h, P->w, P->res, P->p, P->st, P->qflag, P->stageA,
                  P->stageb, P->stagex, P->Ahi, P->Alo, P->SBb, P->cpartB, P->mpart, P->mpartdf, P->mr2part,
                  P->mT, P->mXs, P->mXo, P->mC, P->mG, P->mDY, P->mDYold, P->mZ, P->mH,
                  P->mW, P->mstate, P->tcnt, P->tlmax, P->colexp, P->cshift,
                  P->tptr, P->tsrc, P->cpow, P->Qfix, P->Qbfix, P->lsqr_s, P->W2, P->R2cm,
                  P->R2rm, P->rinv2, P->Dt2, P->vhead2, P->xk, P->xko, P->gk, P->qflag2,
                  P->part2};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (P->st_host) cudaFreeHost(P->st_host);
  if (P->dcol_host) cudaFreeHost(P->dcol_host);
  for (auto &e : P->ev)
    if (e) cudaEventDestroy(e);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  for (auto &e : P->qb.ev)
    if (e) cudaEventDestroy(e);
  if (P->qb.sp) cudaStreamDestroy(P->qb.sp);
  if (P->qb.tws) cudaFree(P->qb.tws);
  for (auto &e : P->chunk_ev)
    if (e) cudaEventDestroy(e);
  if (P->ev_stage) cudaEventDestroy(P->ev_stage);
  if (P->scopy) cudaStreamDestroy(P->scopy);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  if (P->s2) cudaStreamDestroy(P->s2);
  for (auto &e : P->tev) cudaEventDestroy(e);
  delete P;
}

}  // namespace

extern "C" {

void lsq_options_default(lsq_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->zeta = 8;
  o->col_scale = 1;
  o->max_inner = 100;
  o->max_refine = 2;
  o->precision = LSQ_PREC_FP64;
  o->fp32_cond_max = 1e5;
  o->stop_gamma = 10.0;  // Alg. 4 (the Sec. 4.2 text quotes 1 and 0.04)
  o->stop_rho = 0.4;
}

const char *lsq_last_error(void) { return g_err.c_str(); }

lsq_status lsq_plan_create(const lsq_options *opt, void *cuda_stream, lsq_plan *out) {
  if (!out) return fail(LSQ_ERR_INVALID, "out is NULL");
  *out = nullptr;
  LSQ_TRY(validate(opt));
  lsq_plan P = new lsq_plan_s();
  P->s = (cudaStream_t)cuda_stream;
  P->m_cap = opt->m;
  P->n_cap = opt->n;
  P->d_cap = opt->d ? opt->d : (int)(12 * opt->n);
  P->zeta_cap = opt->zeta ? opt->zeta : 8;
  configure_fields(P, opt);
  const int n = (int)P->n;
  cudaError_t e = cudaGetDevice(&P->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->dev);
  if (e != cudaSuccess) {
    free_plan(P);
    return fail(LSQ_ERR_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
  }
  // The pass grid sizes the per-CTA partials.  The CSR passes gather their
  // operands (indices, then the entries they point at) and are bound by load
  // latency, so a sparse plan fills the SMs to the CSR kernel's occupancy
  // limit at 500 columns (5 CTAs: registers), not the dense passes' 2.
  P->gpass = P->nsm * (opt->sparse ? kCsrCtasPerSm : kPassCtasPerSm);
  P->gqr = qr_grid(n + 1, P->nsm);
  // workspace sized for the capacity (equal to the first problem's sizes)
  const size_t nn = (size_t)n * n, dn1 = (size_t)P->d_cap * (n + 1);
  e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(&P->pat_rows, (size_t)P->m_cap * P->zeta_cap));
  A(dalloc(&P->pat_sb, (size_t)P->m));
  if (!opt->sparse && gather_size_ok(P->m_cap, n)) {
    A(dalloc(&P->tcnt, (size_t)P->d_cap));
    A(dalloc(&P->tptr, (size_t)P->d_cap + 1));
    A(dalloc(&P->tsrc, (size_t)P->m_cap * P->zeta_cap));
    A(dalloc(&P->tlmax, 1));
    A(dalloc(&P->colexp, (size_t)P->npad + 1));
    A(dalloc(&P->cshift, (size_t)P->npad + 1));
    A(dalloc(&P->cpow, (size_t)P->npad + 1));
    A(dalloc(&P->Qfix, (size_t)P->m_cap * (size_t)((n + 1) & ~1)));
    A(dalloc(&P->Qbfix, (size_t)P->m_cap));
  }
  P->k = opt->nrhs > 0 ? opt->nrhs : 0;
  A(dalloc(&P->SAb, dn1));
  A(dalloc(&P->W, (size_t)P->d * (n + (P->k > 1 ? P->k : 1))));
  if (P->k > 0) {
    const size_t nk = (size_t)n * P->k, np8k = (size_t)multi_np8(n) * P->k;
    A(dalloc(&P->SBb, (size_t)P->d * (P->k + 1)));
    A(dalloc(&P->cpartB, (size_t)P->gpass * pass_npad(P->k)));
    A(dalloc(&P->mpart, (size_t)P->nsm * np8k));
    A(dalloc(&P->mpartdf, (size_t)P->k * P->gpass * P->npad));
    A(dalloc(&P->mr2part, (size_t)P->nsm * P->k));
    double **mv[] = {&P->mT, &P->mXs, &P->mXo, &P->mC, &P->mG, &P->mDY, &P->mDYold, &P->mZ,
                     &P->mH, &P->mW};
    for (double **v : mv) A(dalloc(v, nk));
    A(dalloc(&P->mstate, 5 * (size_t)P->k));
  }
  A(dalloc(&P->part, (size_t)P->gpass * P->npad));
  A(dalloc(&P->r2part, (size_t)P->gpass));
  A(dalloc(&P->cpart, (size_t)P->gpass * P->npad));
  A(dalloc(&P->dcol, n));
  A(dalloc(&P->dinv, n));
  A(dalloc(&P->Rcm, nn));
  A(dalloc(&P->Rrm, nn));
  A(dalloc(&P->rinv, n));
  A(dalloc(&P->Dt, (size_t)2 * ((n + 31) / 32) * 1024));
  A(dalloc(&P->t, n));
  A(dalloc(&P->vbuf, 2 * (size_t)P->d_cap));
  double **vecs[] = {&P->xs, &P->xo, &P->c, &P->g, &P->dy, &P->dyold, &P->z, &P->h, &P->w, &P->res, &P->p};
  for (double **v : vecs) A(dalloc(v, n));
  A(dalloc(&P->st, 1));
  A(dalloc(&P->qflag, n));
  A(dalloc(&P->lsqr_s, (size_t)P->m_cap));
  A(dalloc(&P->W2, 2 * nn));
  A(dalloc(&P->R2cm, nn));
  A(dalloc(&P->R2rm, nn));
  A(dalloc(&P->rinv2, n));
  A(dalloc(&P->Dt2, (size_t)2 * ((n + 31) / 32) * 1024));
  A(dalloc(&P->vhead2, 4 * (size_t)n));
  A(dalloc(&P->xk, n));
  A(dalloc(&P->xko, n));
  A(dalloc(&P->gk, n));
  A(dalloc(&P->qflag2, n));
  A(dalloc(&P->part2, (size_t)P->gpass * 2 * P->npad));
  A(cudaMallocHost((void **)&P->st_host, sizeof(DevState)));
  A(cudaMallocHost((void **)&P->dcol_host, sizeof(double) * n));
  // hi / lo FP32 planes of A: the double-float inner pass and the FP32 tier read them
  if (!P->o.sparse && (!P->o.inner_fp64_fma || P->o.precision == LSQ_PREC_AUTO ||
                       P->o.precision == LSQ_PREC_FP32_INNER)) {
    A(dalloc(&P->Ahi, (size_t)P->m_cap * ((n + 3) / 4 * 4)));
    A(dalloc(&P->Alo, (size_t)P->m_cap * ((n + 3) / 4 * 4)));
    P->want32 = true;
  }
  for (auto &ev : P->ev) A(cudaEventCreate(&ev));
  A(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
  A(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
  A(cudaStreamCreateWithFlags(&P->s2, cudaStreamNonBlocking));
  {
    int lo = 0, hi = 0;
    A(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    A(cudaStreamCreateWithPriority(&P->qb.sp, cudaStreamNonBlocking, hi));
    for (auto &e : P->qb.ev) A(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    A(dalloc(&P->qb.tws, qr_blocked_tws((int)P->n_cap)));
  }
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    free_plan(P);
    return fail(oom ? LSQ_ERR_OOM : LSQ_ERR_CUDA, std::string("plan allocation: ") + cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(P->st, 0, sizeof(DevState), P->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->qflag, 0, sizeof(int) * (size_t)P->n_cap, P->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->qflag2, 0, sizeof(int) * (size_t)P->n_cap, P->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
  if (e != cudaSuccess) {
    free_plan(P);
    return fail(LSQ_ERR_CUDA, std::string("plan init: ") + cudaGetErrorString(e));
  }
  std::memset(P->st_host, 0, sizeof(DevState));
  *out = P;
  return LSQ_OK;
}

}  // extern "C"

// Re-target a plan within its capacity (used by the request server).
lsq_status lsq::plan_configure(lsq_plan P, const lsq_options *opt) {
  if (!P) return fail(LSQ_ERR_INVALID, "plan is NULL");
  LSQ_TRY(validate(opt));
  const int d = opt->d ? opt->d : (int)(12 * opt->n);
  const int zeta = opt->zeta ? opt->zeta : 8;
  if (opt->m > P->m_cap || opt->n > P->n_cap || d > P->d_cap || zeta > P->zeta_cap)
    return fail(LSQ_ERR_INVALID, "problem exceeds the plan's capacity");
  if ((opt->nrhs > 0) != (P->k > 0) || (P->k > 0 && opt->nrhs != P->k))
    return fail(LSQ_ERR_INVALID, "nrhs differs from the plan's");
  const bool want32 = (opt->precision == LSQ_PREC_AUTO || opt->precision == LSQ_PREC_FP32_INNER);
  if (want32 && !P->Ahi) return fail(LSQ_ERR_INVALID, "plan has no FP32 planes of A");
  configure_fields(P, opt);
  return LSQ_OK;
}

lsq_status lsq::plan_solve(lsq_plan P, int method, const double *dA, const double *db,
                           double *dx, lsq_info *info) {
  if (!P) return fail(LSQ_ERR_INVALID, "plan is NULL");
  return run_solve(P, method, dA, db, dx, info);
}

void lsq::plan_set_stepwise_qr(lsq_plan P, int on) {
  if (P) P->stepwise_qr = on != 0;
}

extern "C" {

void lsq_plan_destroy(lsq_plan plan) { free_plan(plan); }

lsq_status lsq_plan_configure(lsq_plan plan, const lsq_options *opt) {
  return lsq::plan_configure(plan, opt);
}

lsq_status lsq_sketch(lsq_plan plan, const double *dA, const double *db) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  LSQ_TRY(do_sketch(plan, dA, db, false));
  LSQ_TRY(join_condest(plan));
  return read_state(plan);
}

lsq_status lsq_solve_fossils(lsq_plan plan, const double *dA, const double *db, double *dx,
                             lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  return run_solve(plan, 0, dA, db, dx, info);
}

lsq_status lsq_solve_spir(lsq_plan plan, const double *dA, const double *db, double *dx,
                          lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  return run_solve(plan, 1, dA, db, dx, info);
}

lsq_status lsq_solve_spir_lsqr(lsq_plan plan, const double *dA, const double *db, double *dx,
                               lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  return run_solve(plan, 2, dA, db, dx, info);
}

lsq_status lsq_solve_csr(lsq_plan plan, int method, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const double *val, const double *db, double *dx,
                         lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  lsq_plan P = plan;
  if (!P->o.sparse) return fail(LSQ_ERR_INVALID, "the plan was not created with sparse = 1");
  if (!row_ptr || !db || !dx || (nnz > 0 && (!col || !val)))
    return fail(LSQ_ERR_INVALID, "NULL argument");
  if (nnz < 0) return fail(LSQ_ERR_INVALID, "nnz < 0");
  if (method < 0 || method > 2) return fail(LSQ_ERR_INVALID, "method must be 0, 1 or 2");
  P->csr.rp = row_ptr;
  P->csr.col = col;
  P->csr.val = val;
  P->csr.nnz = nnz;
  const lsq_status st = run_solve(P, method, nullptr, db, dx, info);
  P->csr.rp = nullptr;
  P->csr.col = nullptr;
  P->csr.val = nullptr;
  P->csr.nnz = 0;
  return st;
}

lsq_status lsq_solve_complex(lsq_plan plan, int method, const double *dA, int64_t lda,
                             const double *db, double *dx, double *dwork, lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  lsq_plan P = plan;
  if (!dA || !db || !dx || !dwork) return fail(LSQ_ERR_INVALID, "NULL argument");
  if (method < 0 || method > 2) return fail(LSQ_ERR_INVALID, "method must be 0, 1 or 2");
  if (P->m % 2 != 0 || P->n % 2 != 0)
    return fail(LSQ_ERR_INVALID, "a complex solve needs a plan of 2m x 2n (even sizes)");
  if (P->lda != P->n) return fail(LSQ_ERR_INVALID, "a complex solve needs the plan's lda = 2n");
  const int64_t mc = P->m / 2;
  const int nc = (int)(P->n / 2);
  if (lda == 0) lda = nc;
  if (lda < nc) return fail(LSQ_ERR_INVALID, "lda < n");
  if ((reinterpret_cast<uintptr_t>(dA) & 15) != 0 || (reinterpret_cast<uintptr_t>(dwork) & 15) != 0)
    return fail(LSQ_ERR_INVALID, "A and work must be 16-byte aligned");
  LSQ_CU(launch_embed_complex(dA, lda, mc, nc, dwork, P->nsm, P->s));
  return run_solve(P, method, dwork, db, dx, info);
}

lsq_status lsq_solve_fossils_multi(lsq_plan plan, const double *dA, const double *dB,
                                   int64_t ldb, double *dX, lsq_info *info) {
  if (!plan) return fail(LSQ_ERR_INVALID, "plan is NULL");
  return run_solve_multi(plan, dA, dB, ldb, dX, info);
}

lsq_status lsq_solve_host(lsq_plan P, int method, const double *hA, const double *hb, double *hx,
                          lsq_info *info) {
  if (!P) return fail(LSQ_ERR_INVALID, "plan is NULL");
  if (!hA || !hb || !hx) return fail(LSQ_ERR_INVALID, "host buffer is NULL");
  if (method < 0 || method > 2) return fail(LSQ_ERR_INVALID, "method must be 0, 1 or 2");
  const size_t an = (size_t)(P->m - 1) * P->lda + P->n;  // doubles of A read from the host
  if (an > P->stage_cap) {
    if (P->stageA) cudaFree(P->stageA);
    if (P->stageb) cudaFree(P->stageb);
    if (P->stagex) cudaFree(P->stagex);
    P->stageA = P->stageb = P->stagex = nullptr;
    P->stage_cap = 0;
    cudaError_t e = dalloc(&P->stageA, an);
    if (e == cudaSuccess) e = dalloc(&P->stageb, (size_t)P->m_cap);
    if (e == cudaSuccess) e = dalloc(&P->stagex, (size_t)P->n_cap);
    if (e != cudaSuccess) return fail(LSQ_ERR_OOM, "staging allocation failed");
    P->stage_cap = an;
  }
  if (!P->scopy) {
    LSQ_CU(cudaStreamCreateWithFlags(&P->scopy, cudaStreamNonBlocking));
    LSQ_CU(cudaEventCreateWithFlags(&P->ev_stage, cudaEventDisableTiming));
    for (auto &e : P->chunk_ev) LSQ_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  LSQ_TRY(ensure_pattern(P));
  // The gather-form sketch takes A in row chunks of at least kHostChunkBytes,
  // each sketched on the main stream as soon as its copy lands, so the
  // sketch runs under the host-to-device copy of the rest of A.
  const double abytes = 8.0 * (double)an;
  int nch = 1;
  if (P->use_gather)
    nch = (int)std::min<double>(kHostChunksMax, std::floor(abytes / kHostChunkBytes));
  if (nch > 1) {
    // the copies start once the main stream is done with the staging buffers
    LSQ_CU(cudaEventRecord(P->ev_stage, P->s));
    LSQ_CU(cudaStreamWaitEvent(P->scopy, P->ev_stage, 0));
    LSQ_CU(cudaMemcpyAsync(P->stageb, hb, (size_t)P->m * sizeof(double), cudaMemcpyHostToDevice,
                           P->scopy));
    for (int c = 0; c <= nch; c++) P->chunk_row[c] = P->m * c / nch;
    for (int c = 0; c < nch; c++) {
      const int64_t r0 = P->chunk_row[c], r1 = P->chunk_row[c + 1];
      const size_t cnt = (size_t)(r1 - r0 - 1) * P->lda + P->n;
      LSQ_CU(cudaMemcpyAsync(P->stageA + r0 * P->lda, hA + r0 * P->lda, cnt * sizeof(double),
                             cudaMemcpyHostToDevice, P->scopy));
      LSQ_CU(cudaEventRecord(P->chunk_ev[c], P->scopy));
    }
    P->host_chunks = nch;
  } else {
    LSQ_CU(cudaMemcpyAsync(P->stageA, hA, an * sizeof(double), cudaMemcpyHostToDevice, P->s));
    LSQ_CU(cudaMemcpyAsync(P->stageb, hb, (size_t)P->m * sizeof(double), cudaMemcpyHostToDevice,
                           P->s));
  }
  lsq_status st = run_solve(P, method, P->stageA, P->stageb, P->stagex, info);
  P->host_chunks = 0;
  if (st < 0) {
    cudaStreamSynchronize(P->scopy);  // no copy into the staging buffers outlives the call
    return st;
  }
  LSQ_CU(cudaMemcpyAsync(hx, P->stagex, (size_t)P->n * sizeof(double), cudaMemcpyDeviceToHost, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  return st;
}

lsq_status lsq_sketch_pattern(lsq_plan P, int32_t *d_rows, uint32_t *d_signbits) {
  if (!P || !d_rows || !d_signbits) return fail(LSQ_ERR_INVALID, "NULL argument");
  LSQ_TRY(ensure_pattern(P));
  LSQ_CU(cudaMemcpyAsync(d_rows, P->pat_rows, sizeof(int32_t) * (size_t)P->m * P->zeta,
                         cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaMemcpyAsync(d_signbits, P->pat_sb, sizeof(uint32_t) * (size_t)P->m,
                         cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  return LSQ_OK;
}

lsq_status lsq_get_sketch(lsq_plan P, double *dSAb, double *dcolnorm) {
  if (!P) return fail(LSQ_ERR_INVALID, "plan is NULL");
  if (!P->sketched) return fail(LSQ_ERR_INVALID, "call lsq_sketch first");
  // W is overwritten by the QR; the scaled sketch is rebuilt from SAb.
  if (dSAb) {
    const int n = (int)P->n;
    LSQ_CU(launch_sketch_finalize(P->cpart, P->gpass, P->npad, n, P->d, P->zeta, P->o.col_scale,
                                  P->SAb, dSAb, P->dcol, P->dinv, P->st, P->s));
  }
  if (dcolnorm)
    LSQ_CU(cudaMemcpyAsync(dcolnorm, P->dcol, sizeof(double) * P->n, cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  return LSQ_OK;
}

lsq_status lsq_get_sketch_raw(lsq_plan P, double *dSAb) {
  if (!P || !dSAb) return fail(LSQ_ERR_INVALID, "NULL argument");
  if (!P->sketched) return fail(LSQ_ERR_INVALID, "call lsq_sketch first");
  LSQ_CU(cudaMemcpyAsync(dSAb, P->SAb, sizeof(double) * (size_t)P->d * (P->n + 1),
                         cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  return LSQ_OK;
}

lsq_status lsq_get_R(lsq_plan P, double *dR, double *dt, double *dx0, double *condest,
                     double *normest) {
  if (!P) return fail(LSQ_ERR_INVALID, "plan is NULL");
  if (!P->sketched) return fail(LSQ_ERR_INVALID, "call lsq_sketch first");
  const size_t n = (size_t)P->n;
  if (dR) LSQ_CU(cudaMemcpyAsync(dR, P->Rrm, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, P->s));
  if (dt) LSQ_CU(cudaMemcpyAsync(dt, P->t, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->s));
  if (dx0) LSQ_CU(cudaMemcpyAsync(dx0, P->xs, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->s));
  LSQ_CU(cudaStreamSynchronize(P->s));
  if (condest) *condest = P->st_host->condest;
  if (normest) *normest = P->st_host->normest;
  return LSQ_OK;
}

lsq_status lsq_apply_normal(lsq_plan P, const double *dA, const double *dz, double *dh) {
  if (!P || !dA || !dz || !dh) return fail(LSQ_ERR_INVALID, "NULL argument");
  const int n = (int)P->n;
  if (P->sketched && P->use_df && !P->planes_pending)
    LSQ_CU(launch_pass_atax_df(P->Ahi, P->Alo, P->ld32, P->m, n, dz, P->part, P->gpass, P->npad,
                               nullptr, &P->st->err, P->s));
  else if (P->sketched && P->use_eft)
    LSQ_CU(launch_pass_atax_eft(dA, P->lda, P->m, n, dz, P->col_exp, P->part, P->gpass, P->npad,
                                nullptr, P->s));
  else
    LSQ_CU(launch_pass_atax(dA, P->lda, P->m, n, dz, P->part, P->gpass, P->npad, nullptr, P->s));
  LSQ_CU(launch_reduce(P->part, P->gpass, P->npad, n, nullptr, dh, nullptr, nullptr, nullptr, P->s));
  LSQ_TRY(read_state(P));
  return LSQ_OK;
}

lsq_status lsq_apply_normal_multi(lsq_plan P, const double *dA, const double *dZ, double *dH) {
  if (!P || !dA || !dZ || !dH) return fail(LSQ_ERR_INVALID, "NULL argument");
  if (P->k <= 0) return fail(LSQ_ERR_INVALID, "plan was created with nrhs = 0");
  const int n = (int)P->n, k = P->k;
  P->launches = 0;
  if (P->multi_planes && P->use_df) {
    LSQ_CU(launch_multi_df_pass(P, dZ, dH, nullptr, nullptr));
  } else {
    LSQ_CU(launch_multi_atax(dA, P->lda, P->m, n, k, dZ, P->mpart, P->nsm, nullptr, P->s));
    LSQ_CU(launch_multi_reduce(P->mpart, P->nsm, n, k, nullptr, dH, nullptr, nullptr, nullptr,
                               P->s));
  }
  LSQ_TRY(read_state(P));
  return LSQ_OK;
}

lsq_status lsq_sketched_kw(lsq_plan P, const double *dA, const double *db, const double *dx,
                           double *est) {
  if (!P || !dA || !db || !dx || !est) return fail(LSQ_ERR_INVALID, "NULL argument");
  if (P->o.sparse) return fail(LSQ_ERR_INVALID, "the sketched KW estimate needs dense A");
  if (!P->sketched) return fail(LSQ_ERR_INVALID, "call lsq_sketch first");
  const int n = (int)P->n;
  LSQ_CU(launch_scale_vec(n, P->dcol, dx, P->xk, P->s));  // x_s = D x
  LSQ_CU(launch_bnorm2(db, P->m, P->st, P->s));
  LSQ_TRY(kw_eval(P, dA, db, P->xk, dx, false));
  LSQ_TRY(read_state(P));
  *est = P->st_host->kw_est;
  return LSQ_OK;
}

lsq_status lsq_residual(lsq_plan P, const double *dA, const double *db, const double *dx,
                        double *dg, double *r2) {
  if (!P || !dA || !db || !dx || !dg) return fail(LSQ_ERR_INVALID, "NULL argument");
  const int n = (int)P->n;
  LSQ_CU(launch_pass_resid(dA, P->lda, P->m, n, db, dx, P->part, P->r2part, P->gpass, P->npad, P->s));
  LSQ_CU(launch_reduce(P->part, P->gpass, P->npad, n, nullptr, dg, P->r2part, &P->st->r2, nullptr, P->s));
  LSQ_TRY(read_state(P));
  if (r2) *r2 = P->st_host->r2;
  return LSQ_OK;
}

lsq_status lsq_trsv(lsq_plan P, int trans, const double *dy, double *dx) {
  if (!P || !dy || !dx) return fail(LSQ_ERR_INVALID, "NULL argument");
  if (!P->sketched) return fail(LSQ_ERR_INVALID, "call lsq_sketch first");
  LSQ_CU(launch_trsv(P->Rcm, P->Rrm, P->rinv, P->Dt, (int)P->n, trans ? 1 : 0, dy, nullptr, dx, nullptr,
                     nullptr, nullptr, nullptr, nullptr, P->s, 1, 0,
                       &P->st->err));
  LSQ_CU(cudaStreamSynchronize(P->s));
  return LSQ_OK;
}

}  // extern "C"

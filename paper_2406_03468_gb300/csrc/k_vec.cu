// n-vector steps of the inner solvers, one CTA each (n <= LSQ_MAX_N):
//   Polyak heavy ball (Alg. 5, in the loop form of Alg. 4):
//     Delta = alpha (c - M dy) + beta (dy - dy_old);  (dy, dy_old) <- (dy + Delta, dy)
//   conjugate gradient on M dy = c from dy = 0 (Alg. 3's inner solver)
// and the step-1 stopping rule of Sec. 4.2 ("Adaptive stopping", item 1):
//   stop once ||Delta|| <= u (gamma normest ||x_0|| + rho condest ||b - A x_0||).
// The stop decision is taken on the device (DevState::done) so that the
// host never waits between iterations.
#include <algorithm>

#include "lsq_common.cuh"

namespace lsq {

namespace {

__device__ void inner_init_body(int method, int n, const double *__restrict__ c, double *dy,
                                double *dy_old, double *res, double *p, int max_iters,
                                int use_thresh, DevState *st) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ci = c[i];
    if (method == 0) {
      dy[i] = ci;
      dy_old[i] = ci;
    } else {
      dy[i] = 0.0;
      res[i] = ci;
      p[i] = ci;
      s = fma(ci, ci, s);
    }
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) {
    st->rho = s;
    st->iters = 0;
    st->max_iters = max_iters;
    st->use_thresh = use_thresh;
    st->dnorm2 = 0.0;
    // CG with c = 0 (rho = 0) has dy = 0 exactly and no update to make: its
    // first step would be 0 / 0
    st->done = (max_iters <= 0 || (method != 0 && !(s > 0.0))) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(kVecThreads)
    inner_init_kernel(int method, int n, const double *__restrict__ c, double *dy,
                      double *dy_old, double *res, double *p, int max_iters, int use_thresh,
                      DevState *st) {
  inner_init_body(method, n, c, dy, dy_old, res, p, max_iters, use_thresh, st);
}

__device__ __forceinline__ void finish_update(DevState *st, double dn2, bool exhausted) {
  const int it = st->iters + 1;
  st->iters = it;
  st->dnorm2 = dn2;
  bool stop = it >= st->max_iters || exhausted;
  if (st->use_thresh && sqrt(dn2) <= st->thresh1) stop = true;
  if (stop) st->done = 1;
}

__device__ void polyak_body(int n, const double *__restrict__ c, const double *__restrict__ w,
                            double *dy, double *dy_old, DevState *st) {
  __shared__ double scratch[32];
  const double alpha = st->alpha, beta = st->beta;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double y = dy[i];
    const double delta = alpha * (c[i] - w[i]) + beta * (y - dy_old[i]);
    dy_old[i] = y;
    dy[i] = y + delta;
    s = fma(delta, delta, s);
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) finish_update(st, s, false);
}

__global__ void __launch_bounds__(kVecThreads)
    polyak_update_kernel(int n, const double *__restrict__ c, const double *__restrict__ w,
                         double *dy, double *dy_old, DevState *st) {
  if (*(volatile int *)&st->done) return;
  polyak_body(n, c, w, dy, dy_old, st);
}

__device__ void cg_body(int n, const double *__restrict__ q, double *p, double *res, double *dy,
                        DevState *st) {
  __shared__ double scratch[32];
  double pq = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) pq = fma(p[i], q[i], pq);
  pq = block_sum(pq, scratch);
  const double rho = st->rho;
  const double gam = rho / pq;
  double rr = 0.0, ss = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double step = gam * p[i];
    dy[i] += step;
    const double r = res[i] - gam * q[i];
    res[i] = r;
    rr = fma(r, r, rr);
    ss = fma(step, step, ss);
  }
  rr = block_sum(rr, scratch);
  ss = block_sum(ss, scratch);
  const double bet = rr / rho;
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = res[i] + bet * p[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    st->rho = rr;
    finish_update(st, ss, !(rr > 0.0));
  }
}

__global__ void __launch_bounds__(kVecThreads)
    cg_update_kernel(int n, const double *__restrict__ q, double *p, double *res, double *dy,
                     DevState *st) {
  if (*(volatile int *)&st->done) return;
  cg_body(n, q, p, res, dy, st);
}

// Batched forms (one CTA per item, lsq_batch.cu).  b_init: at step 0 the
// step-1 threshold (as set_thresh) and the cap max_inner with the threshold
// test; at step 1 the cap q2 (set by b_setup from condest), no threshold.
__global__ void __launch_bounds__(kVecThreads)
    b_init_kernel(const BItem *__restrict__ items, int step, int max_inner, double gamma,
                  double rho) {
  const BItem &it = items[blockIdx.x];
  DevState *st = it.st;
  if (threadIdx.x == 0 && step == 0)
    st->thresh1 = kU * (gamma * st->normest * sqrt(st->x0norm2) + rho * st->condest * sqrt(st->r2));
  __syncthreads();
  const int cap = step == 0 ? max_inner : st->q2;
  inner_init_body(it.method, it.n, it.c, it.dy, it.dyold, it.res, it.p, cap, step == 0 ? 1 : 0,
                  st);
}

__global__ void __launch_bounds__(kVecThreads) b_update_kernel(const BItem *__restrict__ items) {
  const BItem &it = items[blockIdx.x];
  if (*(volatile int *)&it.st->done) return;
  if (it.method == 0) polyak_body(it.n, it.c, it.w, it.dy, it.dyold, it.st);
  else cg_body(it.n, it.w, it.p, it.res, it.dy, it.st);
}

__global__ void b_copy_x_kernel(const BItem *__restrict__ items) {
  const BItem &it = items[blockIdx.x];
  for (int i = threadIdx.x; i < it.n; i += blockDim.x) it.x[i] = it.xo[i];
}

// ||b||^2 on one CTA (a fixed order).
__global__ void __launch_bounds__(kVecThreads)
    bnorm2_kernel(const double *__restrict__ b, int64_t m, DevState *st) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma(b[i], b[i], s);
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) st->bnorm2 = s;
}

// The stacked matrix of the sketched Karlson-Walden estimate (eq. (sketched-
// kw)): (SA)^T (SA) + lam I = R^T R + lam I = R_lam^T R_lam with R_lam the R
// factor of [R; sqrt(lam) I], so the estimate is the prefactor times
// ||R_lam^-T A^T r|| -- the value Alg. 4 computes through the SVD of SA.
// theta = ||A D^-1||_F / ||b|| on the column-scaled problem (Sec. 4.2).
__global__ void kw_build_kernel(const double *__restrict__ Rcm, int n,
                                const double *__restrict__ dcol, const double *__restrict__ dinv,
                                const double *__restrict__ xs, double *__restrict__ W2,
                                DevState *st) {
  __shared__ double scratch[32];
  __shared__ double s_lam;
  double a2 = 0.0, x2 = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double c = dcol[j] * dinv[j];
    a2 = fma(c, c, a2);
    x2 = fma(xs[j], xs[j], x2);
  }
  a2 = block_sum(a2, scratch);
  x2 = block_sum(x2, scratch);
  if (threadIdx.x == 0) {
    const double th2 = a2 / st->bnorm2;
    const double den = 1.0 + th2 * x2;
    if (blockIdx.x == 0) st->kw_xn2 = x2;
    s_lam = th2 * st->kw_r2 / den;
    st->kw_pref = sqrt(th2) / sqrt(den);
  }
  __syncthreads();
  const double sl = sqrt(s_lam);
  const int d2 = 2 * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)d2 * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / d2), i = (int)(idx % d2);
    double v;
    if (i < n) v = (i <= j) ? Rcm[(size_t)j * n + i] : 0.0;
    else v = (i - n == j) ? sl : 0.0;
    W2[idx] = v;
  }
}

__global__ void kw_finish_kernel(DevState *st) { st->kw_est = st->kw_pref * sqrt(st->kw_y2); }

__global__ void scale_vec_kernel(int n, const double *__restrict__ sc, const double *__restrict__ x,
                                 double *__restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = sc[i] * x[i];
}

__global__ void set_thresh_kernel(double gamma, double rho, DevState *st) {
  st->thresh1 = kU * (gamma * st->normest * sqrt(st->x0norm2) + rho * st->condest * sqrt(st->r2));
}

}  // namespace

cudaError_t launch_inner_init(int method, int n, const double *c, double *dy, double *dy_old,
                              double *res, double *p, int max_iters, int use_thresh,
                              DevState *st, cudaStream_t s) {
  inner_init_kernel<<<1, kVecThreads, 0, s>>>(method, n, c, dy, dy_old, res, p, max_iters,
                                              use_thresh, st);
  return cudaGetLastError();
}

cudaError_t launch_polyak_update(int n, const double *c, const double *w, double *dy,
                                 double *dy_old, DevState *st, cudaStream_t s) {
  polyak_update_kernel<<<1, kVecThreads, 0, s>>>(n, c, w, dy, dy_old, st);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(int n, const double *q, double *p, double *res, double *dy,
                             DevState *st, cudaStream_t s) {
  cg_update_kernel<<<1, kVecThreads, 0, s>>>(n, q, p, res, dy, st);
  return cudaGetLastError();
}

cudaError_t launch_b_init(const BItem *items, int count, int step, int max_inner, double gamma,
                          double rho, cudaStream_t s) {
  b_init_kernel<<<count, kVecThreads, 0, s>>>(items, step, max_inner, gamma, rho);
  return cudaGetLastError();
}

cudaError_t launch_b_update(const BItem *items, int count, cudaStream_t s) {
  b_update_kernel<<<count, kVecThreads, 0, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_b_copy_x(const BItem *items, int count, cudaStream_t s) {
  b_copy_x_kernel<<<count, 256, 0, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_bnorm2(const double *b, int64_t m, DevState *st, cudaStream_t s) {
  bnorm2_kernel<<<1, kVecThreads, 0, s>>>(b, m, st);
  return cudaGetLastError();
}

cudaError_t launch_kw_build(const double *Rcm, int n, const double *dcol, const double *dinv,
                            const double *xs, double *W2, DevState *st, cudaStream_t s) {
  // every CTA computes lam (the same value) for its share of W2
  const int64_t cnt = 2 * (int64_t)n * n;
  const int grid = (int)std::min<int64_t>(64, (cnt + 1023) / 1024);
  kw_build_kernel<<<grid, 1024, 0, s>>>(Rcm, n, dcol, dinv, xs, W2, st);
  return cudaGetLastError();
}

cudaError_t launch_kw_finish(DevState *st, cudaStream_t s) {
  kw_finish_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

cudaError_t launch_scale_vec(int n, const double *sc, const double *x, double *y, cudaStream_t s) {
  scale_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, sc, x, y);
  return cudaGetLastError();
}

cudaError_t launch_set_thresh(double gamma, double rho, DevState *st, cudaStream_t s) {
  set_thresh_kernel<<<1, 1, 0, s>>>(gamma, rho, st);
  return cudaGetLastError();
}

}  // namespace lsq

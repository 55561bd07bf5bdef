// Householder QR of the scaled sketch [SA Sb] (d x (n+1), column-major,
// leading dimension d), giving R (the preconditioner, Sec. 2.1) in the upper
// triangle and t = (Q^T Sb)[0:n] in the last column (the augmented column of
// Alg. 1's sketch-and-solve start).  The paper's analysis assumes Householder
// QR (Lemma 6.3), so this is plain column-by-column Householder:
//   v = x + sign(x_1) ||x|| e_1,  v <- v / ||v||,  A <- A - 2 v (v^T A),
// with ||v|| from the identity ||v||^2 = 2 ||x|| (||x|| + |x_1|) and v scaled
// by the reciprocal 1/||v|| (one rounding more per entry than a division; the
// FP64 divide runs on GB300's narrow FP64 pipe and dominated the step).
//
// GB300 design: one persistent cooperative launch, one CTA per SM.  Column
// j belongs to CTA j mod G for the whole factorisation and, when the CTA's
// columns fit (d = 12n up to n ~ 600), lives in that CTA's shared memory
// from start to end.  Step k: every CTA applies H_k (v_k from one of two
// global buffers, alternating with the parity of k) to its columns j > k;
// the owner of column k+1 does that column first and then builds v_{k+1}
// into the other buffer (lookahead), so no CTA waits for a serial reflector
// step; one bounded grid barrier closes the step.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kQrThreads = 512;
constexpr int kQrBatch = 8;  // columns updated together by one CTA

// Householder vector of column `col` at step k (col holds rows 0..d-1, the
// entries below row k are the current trailing column): writes
// v = (x + sign(x_k)||x|| e_k) / ||v|| to v[k..d-1] and R_kk = -sign(x_k)||x||
// to col[k].  Whole CTA.
__device__ void make_reflector(double *col, int k, int d, double *v, double *red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double s = 0.0;
  for (int i = k + tid; i < d; i += nt) s = fma(col[i], col[i], s);
  s = block_sum(s, red);
  const double nx = sqrt(s);
  const double x0 = col[k];
  const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
  const double v0 = x0 + sg * nx;
  // ||v||^2 = ||x||^2 - x0^2 + (x0 + sign(x0) ||x||)^2 = 2 ||x|| (||x|| + |x0|)
  const double nv = sqrt(2.0 * nx * (nx + fabs(x0)));
  const double inv = (nv > 0.0) ? 1.0 / nv : 0.0;
  for (int i = k + tid; i < d; i += nt) v[i] = ((i == k) ? v0 : col[i]) * inv;
  __syncthreads();
  if (tid == 0) col[k] = -sg * nx;
}

// Apply H_k = I - 2 v v^T (v from global memory, rows k..d-1) to `cnt` <= kQrBatch
// columns cols[0..cnt).  Whole CTA.
__device__ void apply_reflector(double *const *cols, int cnt, int k, int d, const double *v,
                                double *red, double *wsh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double acc[kQrBatch];
#pragma unroll
  for (int c = 0; c < kQrBatch; c++) acc[c] = 0.0;
  for (int i = k + tid; i < d; i += nt) {
    const double vi = __ldcg(v + i);
#pragma unroll
    for (int c = 0; c < kQrBatch; c++)
      if (c < cnt) acc[c] = fma(vi, cols[c][i], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < kQrBatch; c++)
    if (c < cnt) acc[c] = warp_sum(acc[c]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kQrBatch; c++)
      if (c < cnt) red[warp * kQrBatch + c] = acc[c];
  }
  __syncthreads();
  if (tid < cnt) {
    double sacc = 0.0;
    for (int w = 0; w < nw; w++) sacc += red[w * kQrBatch + tid];
    wsh[tid] = 2.0 * sacc;
  }
  __syncthreads();
  for (int i = k + tid; i < d; i += nt) {
    const double vi = __ldcg(v + i);
#pragma unroll
    for (int c = 0; c < kQrBatch; c++)
      if (c < cnt) cols[c][i] = fma(-wsh[c], vi, cols[c][i]);
  }
  __syncthreads();
}

// SMEM: the CTA's columns live in shared memory for the whole factorisation.
template <bool SMEM>
__global__ void __launch_bounds__(kQrThreads, 1)
    qr_kernel(double *__restrict__ W, int d, int n, int ncols, double *__restrict__ vbuf,
              unsigned int *bar, DevState *st, uint64_t timeout_ns) {
  extern __shared__ double dsm[];
  __shared__ double red[kQrThreads / 32 * kQrBatch];
  __shared__ double wsh[kQrBatch];
  const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int nloc = (ncols - me + G - 1) / G;  // local columns j = me + l G
  auto colp = [&](int l) -> double * {
    return SMEM ? dsm + (size_t)l * d : W + (size_t)(me + l * G) * d;
  };
  if (SMEM) {
    for (int l = 0; l < nloc; l++)
      for (int i = tid; i < d; i += nt) dsm[(size_t)l * d + i] = W[(size_t)(me + l * G) * d + i];
    __syncthreads();
  }
  if (me == 0) make_reflector(colp(0), 0, d, vbuf, red);
  if (!grid_barrier(bar, bar + 1, &st->err, timeout_ns)) return;
  double *cols[kQrBatch];
  for (int k = 0; k < n; k++) {
    const double *v = vbuf + (size_t)(k & 1) * d;
    const int l0 = (k + 1 > me) ? (k + 1 - me + G - 1) / G : 0;  // first local column > k
    int l = l0;
    // Lookahead: the owner of column k+1 applies H_k to it first and builds
    // v_{k+1} into the other buffer while the rest of the grid is updating.
    if (k + 1 < n && (k + 1) % G == me && l < nloc) {
      cols[0] = colp(l);
      apply_reflector(cols, 1, k, d, v, red, wsh);
      make_reflector(colp(l), k + 1, d, vbuf + (size_t)((k + 1) & 1) * d, red);
      l++;
    }
    while (l < nloc) {
      int cnt = 0;
      for (; cnt < kQrBatch && l < nloc; cnt++, l++) cols[cnt] = colp(l);
      apply_reflector(cols, cnt, k, d, v, red, wsh);
    }
    if (!grid_barrier(bar, bar + 1, &st->err, timeout_ns)) return;
  }
  if (SMEM) {
    for (int l2 = 0; l2 < nloc; l2++)
      for (int i = tid; i < d; i += nt) W[(size_t)(me + l2 * G) * d + i] = dsm[(size_t)l2 * d + i];
  }
}

// Non-cooperative form for concurrent solves (served requests): one launch
// per column step, the kernel boundary acting as the grid barrier.  Same
// column ownership (j mod G), same lookahead, columns in global memory.
__global__ void __launch_bounds__(kQrThreads)
    qr_step_kernel(double *__restrict__ W, int d, int n, int ncols, double *__restrict__ vbuf,
                   int k) {
  __shared__ double red[kQrThreads / 32 * kQrBatch];
  __shared__ double wsh[kQrBatch];
  const int G = gridDim.x, me = blockIdx.x;
  const int nloc = (ncols - me + G - 1) / G;
  auto colp = [&](int l) -> double * { return W + (size_t)(me + l * G) * d; };
  if (k < 0) {  // prologue: v_0
    if (me == 0) make_reflector(colp(0), 0, d, vbuf, red);
    return;
  }
  const double *v = vbuf + (size_t)(k & 1) * d;
  double *cols[kQrBatch];
  const int l0 = (k + 1 > me) ? (k + 1 - me + G - 1) / G : 0;
  int l = l0;
  if (k + 1 < n && (k + 1) % G == me && l < nloc) {
    cols[0] = colp(l);
    apply_reflector(cols, 1, k, d, v, red, wsh);
    make_reflector(colp(l), k + 1, d, vbuf + (size_t)((k + 1) & 1) * d, red);
    l++;
  }
  while (l < nloc) {
    int cnt = 0;
    for (; cnt < kQrBatch && l < nloc; cnt++, l++) cols[cnt] = colp(l);
    apply_reflector(cols, cnt, k, d, v, red, wsh);
  }
}

__global__ void extract_r_kernel(const double *__restrict__ W, int d, int n, int nb, double *Rcm,
                                 double *Rrm, double *rinv, double *t) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  if (idx < nn) {
    const int j = (int)(idx / n), i = (int)(idx % n);  // column j, row i
    const double v = (i <= j) ? W[(size_t)j * d + i] : 0.0;
    Rcm[(size_t)j * n + i] = v;
    Rrm[(size_t)i * n + j] = v;
  }
  if (idx < n) rinv[idx] = 1.0 / W[(size_t)idx * d + idx];
  // t (n x nb, column-major) = rows 0..n-1 of the augmented columns
  if (idx < (int64_t)n * nb) {
    const int c = (int)(idx / n), i = (int)(idx % n);
    t[idx] = W[(size_t)(n + c) * d + i];
  }
}

}  // namespace

int qr_grid(int ncols, int nsm) { return ncols < nsm ? ncols : nsm; }

// Largest dynamic shared memory the columns may use (227 KB opt-in minus the static part).
constexpr size_t kQrSmemMax = 225 * 1024;

cudaError_t launch_qr(double *W, int d, int n, int ncols, double *vbuf, unsigned int *bar,
                      DevState *st, int grid, uint64_t timeout_ns, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void *args[] = {&W, &d, &n, &ncols, &vbuf, &bar, &st, &timeout_ns};
  const int nloc_max = (ncols + grid - 1) / grid;
  const size_t smem = (size_t)nloc_max * d * sizeof(double);
  if (smem <= kQrSmemMax) {
    e = cudaFuncSetAttribute((const void *)qr_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)qr_kernel<true>, dim3(grid),
                                       dim3(kQrThreads), args, smem, s);
  }
  return cudaLaunchCooperativeKernel((const void *)qr_kernel<false>, dim3(grid), dim3(kQrThreads),
                                     args, 0, s);
}

cudaError_t launch_qr_stepwise(double *W, int d, int n, int ncols, double *vbuf, int grid,
                               cudaStream_t s) {
  for (int k = -1; k < n; k++) {
    qr_step_kernel<<<grid, kQrThreads, 0, s>>>(W, d, n, ncols, vbuf, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_extract_r(const double *W, int d, int n, int nb, double *Rcm, double *Rrm,
                             double *rinv, double *t, cudaStream_t s) {
  const int64_t nn = (int64_t)n * (n > nb ? n : nb);
  const int th = 256;
  extract_r_kernel<<<(unsigned)((nn + th - 1) / th), th, 0, s>>>(W, d, n, nb, Rcm, Rrm, rinv, t);
  return cudaGetLastError();
}

}  // namespace lsq

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
// GB300 design: one persistent cooperative launch.  Column j belongs to CTA
// j mod G for the whole factorisation, so its data stays with one SM (the
// L1 of that SM never holds another CTA's column).  Step k: the owner of
// column k forms v_k into one of two global buffers (alternating by the
// parity of k), one bounded grid barrier, then every CTA applies H_k to the
// columns it owns.  One barrier per column; the double buffer keeps the
// owner of column k+1 from overwriting v_k while others still read it.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kQrThreads = 512;
constexpr int kQrBatch = 8;  // columns updated together by one CTA

__global__ void __launch_bounds__(kQrThreads, 1)
    qr_kernel(double *__restrict__ W, int d, int n, double *__restrict__ vbuf,
              unsigned int *bar, DevState *st, uint64_t timeout_ns) {
  __shared__ double red[kQrThreads / 32 * kQrBatch];
  __shared__ double wsh[kQrBatch];
  const int G = gridDim.x, me = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int ncols = n + 1;
  for (int k = 0; k < n; k++) {
    double *v = vbuf + (size_t)(k & 1) * d;
    __syncthreads();
    if (k % G == me) {
      double *col = W + (size_t)k * d;
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
      for (int i = k + tid; i < d; i += nt) col[i] = (i == k) ? -sg * nx : 0.0;
    }
    if (!grid_barrier(bar, bar + 1, &st->err, timeout_ns)) return;
    // Apply H_k to the owned columns j > k (the augmented column n included).
    const int jf = k + 1 + (((me - (k + 1)) % G) + G) % G;
    for (int jb = jf; jb < ncols; jb += G * kQrBatch) {
      double acc[kQrBatch];
#pragma unroll
      for (int c = 0; c < kQrBatch; c++) acc[c] = 0.0;
      for (int i = k + tid; i < d; i += nt) {
        const double vi = __ldcg(v + i);
#pragma unroll
        for (int c = 0; c < kQrBatch; c++) {
          const int j = jb + c * G;
          if (j < ncols) acc[c] = fma(vi, W[(size_t)j * d + i], acc[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < kQrBatch; c++) acc[c] = warp_sum(acc[c]);
      __syncthreads();
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < kQrBatch; c++) red[warp * kQrBatch + c] = acc[c];
      }
      __syncthreads();
      if (tid < kQrBatch) {
        double sacc = 0.0;
        for (int w = 0; w < nw; w++) sacc += red[w * kQrBatch + tid];
        wsh[tid] = 2.0 * sacc;
      }
      __syncthreads();
      for (int i = k + tid; i < d; i += nt) {
        const double vi = __ldcg(v + i);
#pragma unroll
        for (int c = 0; c < kQrBatch; c++) {
          const int j = jb + c * G;
          if (j < ncols) {
            double *p = W + (size_t)j * d + i;
            *p = fma(-wsh[c], vi, *p);
          }
        }
      }
    }
  }
}

__global__ void extract_r_kernel(const double *__restrict__ W, int d, int n, double *Rcm,
                                 double *Rrm, double *rinv, double *t) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  if (idx < nn) {
    const int j = (int)(idx / n), i = (int)(idx % n);  // column j, row i
    const double v = (i <= j) ? W[(size_t)j * d + i] : 0.0;
    Rcm[(size_t)j * n + i] = v;
    Rrm[(size_t)i * n + j] = v;
  }
  if (idx < n) {
    rinv[idx] = 1.0 / W[(size_t)idx * d + idx];
    t[idx] = W[(size_t)n * d + idx];
  }
}

}  // namespace

int qr_grid(int n, int nsm) { return (n + 1) < nsm ? (n + 1) : nsm; }

cudaError_t launch_qr(double *W, int d, int n, double *vbuf, unsigned int *bar, DevState *st,
                      int grid, uint64_t timeout_ns, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  void *args[] = {&W, &d, &n, &vbuf, &bar, &st, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void *)qr_kernel, dim3(grid), dim3(kQrThreads), args,
                                     0, s);
}

cudaError_t launch_extract_r(const double *W, int d, int n, double *Rcm, double *Rrm,
                             double *rinv, double *t, cudaStream_t s) {
  const int64_t nn = (int64_t)n * n;
  const int th = 256;
  extract_r_kernel<<<(unsigned)((nn + th - 1) / th), th, 0, s>>>(W, d, n, Rcm, Rrm, rinv, t);
  return cudaGetLastError();
}

}  // namespace lsq

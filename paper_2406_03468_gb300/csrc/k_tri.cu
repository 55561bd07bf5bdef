// Triangular solves with the preconditioner R by back substitution (the
// analysis computes every R^{-1} z and R^{-T} z this way: Sec. 6, notation,
// and Proposition 6.5), and the condest / normest estimates of R that the
// step-1 stopping rule and the q0 count use (Sec. 4.2; Alg. 4 reads them off
// the SVD of SA, whose singular values equal those of R).
//
// One CTA per solve: the vector lives in shared memory; R (n x n) is read
// from L2 in both layouts so that every access is coalesced -- column j of R
// (column-major copy) for R x = y, row j of R (row-major copy) for R^T x = y.
// Blocked by 32: warp 0 solves each 32 x 32 diagonal block with shuffles,
// then the whole CTA subtracts the block's contribution from the rest, so a
// solve costs ceil(n/32) block barriers.  x_j = y_j * (1 / R_jj) with the
// reciprocals computed once per factorisation; that perturbs each diagonal
// entry by at most two roundings, so the solve stays backward stable.
#include "lsq_common.cuh"

namespace lsq {

namespace {

// tile: 32 x 33 doubles of shared memory for the diagonal block.
__device__ void block_trsv(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                           const double *__restrict__ rinv, int n, int trans, double *sy,
                           double *tile) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nt = blockDim.x;
  const int nb = (n + 31) / 32;
  for (int bb = 0; bb < nb; bb++) {
    const int blk = trans ? bb : nb - 1 - bb;
    const int j0 = blk * 32, j1 = min(n, j0 + 32), len = j1 - j0;
    // stage the diagonal block: tile[jj][l] = column jj (trans 0) / row jj (trans 1) entry l
    const double *src = trans ? Rrm : Rcm;
    for (int e = threadIdx.x; e < 32 * 32; e += nt) {
      const int jj = e >> 5, l = e & 31;
      tile[jj * 33 + l] = (jj < len && l < len) ? src[(size_t)(j0 + jj) * n + j0 + l] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double yl = (lane < len) ? sy[j0 + lane] : 0.0;
      const double ri = (lane < len) ? rinv[j0 + lane] : 0.0;
      if (!trans) {
        for (int jj = len - 1; jj >= 0; jj--) {
          const double xj = __shfl_sync(0xffffffffu, yl * ri, jj);
          if (lane == jj) yl = xj;
          else if (lane < jj) yl = fma(-tile[jj * 33 + lane], xj, yl);
        }
      } else {
        for (int jj = 0; jj < len; jj++) {
          const double xj = __shfl_sync(0xffffffffu, yl * ri, jj);
          if (lane == jj) yl = xj;
          else if (lane > jj && lane < len) yl = fma(-tile[jj * 33 + lane], xj, yl);
        }
      }
      if (lane < len) sy[j0 + lane] = yl;
    }
    __syncthreads();
    // Remaining rows: subtract this block's contribution.  Four independent
    // accumulators per row keep the FP64 FMA chains short (the FP64 pipe's
    // latency, not its throughput, bounds a one-CTA solve).
    const double *Rb = trans ? Rrm : Rcm;
    const int ib = trans ? j1 : 0, ie = trans ? n : j0;
    for (int i = ib + threadIdx.x; i < ie; i += nt) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int j = j0;
      for (; j + 3 < j1; j += 4) {
        a0 = fma(Rb[(size_t)j * n + i], sy[j], a0);
        a1 = fma(Rb[(size_t)(j + 1) * n + i], sy[j + 1], a1);
        a2 = fma(Rb[(size_t)(j + 2) * n + i], sy[j + 2], a2);
        a3 = fma(Rb[(size_t)(j + 3) * n + i], sy[j + 3], a3);
      }
      for (; j < j1; j++) a0 = fma(Rb[(size_t)j * n + i], sy[j], a0);
      sy[i] -= (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads)
    trsv_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                const double *__restrict__ rinv, int n, int trans, const double *y,
                const double *in_scale, double *out, const double *out_scale, double *out_scaled,
                double *accum, double *norm2_out, const DevState *gate, int64_t bstride) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  // batched: CTA b solves the b-th vector of each operand (offset b * bstride)
  const int64_t off = (int64_t)blockIdx.x * bstride;
  y += off;
  if (out) out += off;
  if (out_scaled) out_scaled += off;
  if (accum) accum += off;
  if (norm2_out) norm2_out += blockIdx.x;
  extern __shared__ double sy[];
  double *scratch = sy + n;
  double *tile = scratch + 32;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    sy[i] = in_scale ? y[i] * in_scale[i] : y[i];
  __syncthreads();
  block_trsv(Rcm, Rrm, rinv, n, trans, sy, tile);
  double nrm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double x = sy[i];
    if (accum) {
      x = accum[i] + x;
      accum[i] = x;
    }
    if (out) out[i] = x;
    if (out_scaled) out_scaled[i] = out_scale[i] * x;
    nrm = fma(x, x, nrm);
  }
  if (norm2_out) {
    nrm = block_sum(nrm, scratch);
    if (threadIdx.x == 0) *norm2_out = nrm;
  }
}

// y = R v (upper, via the column-major copy) or y = R^T v (via the row-major copy).
__device__ void block_trmv(const double *__restrict__ Rcm, const double *__restrict__ Rrm, int n,
                           int trans, const double *sv, double *sy) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double acc = 0.0;
    if (!trans) {
      for (int j = i; j < n; j++) acc = fma(Rcm[(size_t)j * n + i], sv[j], acc);
    } else {
      for (int j = 0; j <= i; j++) acc = fma(Rrm[(size_t)j * n + i], sv[j], acc);
    }
    sy[i] = acc;
  }
  __syncthreads();
}

__device__ double block_normalize(double *sv, int n, double *scratch) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(sv[i], sv[i], s);
  s = sqrt(block_sum(s, scratch));
  const double inv = (s > 0.0) ? 1.0 / s : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sv[i] *= inv;
  __syncthreads();
  return s;
}

// sigma_max(R) by power iteration on R^T R and sigma_min(R) by inverse power
// iteration on (R^T R)^{-1}, from a fixed start vector.
__global__ void __launch_bounds__(kVecThreads)
    condest_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                   const double *__restrict__ rinv, int n, int iters, DevState *st) {
  extern __shared__ double sm[];
  double *v = sm, *y = sm + n, *scratch = sm + 2 * n, *tile = scratch + 32;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.0 + 0.25 * (double)((i * 7919) % 17);
  __syncthreads();
  block_normalize(v, n, scratch);
  double smax = 0.0;
  for (int it = 0; it < iters; it++) {
    block_trmv(Rcm, Rrm, n, 0, v, y);
    block_trmv(Rcm, Rrm, n, 1, y, v);
    block_normalize(v, n, scratch);
  }
  block_trmv(Rcm, Rrm, n, 0, v, y);
  smax = block_normalize(y, n, scratch);

  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = 1.0 + 0.25 * (double)((i * 104729) % 13);
  __syncthreads();
  block_normalize(v, n, scratch);
  double winv = 0.0;
  for (int it = 0; it <= iters; it++) {
    block_trsv(Rcm, Rrm, rinv, n, 1, v, tile);  // v <- R^{-T} v
    winv = block_normalize(v, n, scratch);
    if (it == iters) break;
    block_trsv(Rcm, Rrm, rinv, n, 0, v, tile);  // v <- R^{-1} v
    block_normalize(v, n, scratch);
  }
  if (threadIdx.x == 0) {
    const double smin = (winv > 0.0) ? 1.0 / winv : 0.0;
    st->normest = smax;
    st->condest = (smin > 0.0) ? smax / smin : INFINITY;
  }
}

}  // namespace

cudaError_t launch_trsv(const double *Rcm, const double *Rrm, const double *rinv, int n, int trans,
                        const double *y, const double *in_scale, double *out,
                        const double *out_scale, double *out_scaled, double *accum,
                        double *norm2_out, const DevState *gate, cudaStream_t s, int batch,
                        int64_t bstride) {
  const size_t smem = (size_t)(n + 32 + 32 * 33) * sizeof(double);
  trsv_kernel<<<batch, kVecThreads, smem, s>>>(Rcm, Rrm, rinv, n, trans, y, in_scale, out,
                                               out_scale, out_scaled, accum, norm2_out, gate,
                                               bstride);
  return cudaGetLastError();
}

cudaError_t launch_condest(const double *Rcm, const double *Rrm, const double *rinv, int n,
                           int iters, DevState *st, cudaStream_t s) {
  const size_t smem = (size_t)(2 * n + 32 + 32 * 33) * sizeof(double);
  condest_kernel<<<1, kVecThreads, smem, s>>>(Rcm, Rrm, rinv, n, iters, st);
  return cudaGetLastError();
}

}  // namespace lsq

// Triangular solves with the preconditioner R by back substitution (the
// analysis computes every R^{-1} z and R^{-T} z this way: Sec. 6, notation,
// and Proposition 6.5), and the condest / normest estimates of R that the
// step-1 stopping rule and the q0 count use (Sec. 4.2; Alg. 4 reads them off
// the SVD of SA, whose singular values equal those of R).
//
// One CTA per solve: the vector lives in shared memory; R (n x n) is read
// from L2 in both layouts so that every access is coalesced -- column j of R
// (column-major copy) for R x = y, row j of R (row-major copy) for R^T x = y.
// Blocked by 16: warp 0 solves each 16 x 16 diagonal block with shuffles,
// then the whole CTA (one thread per row) subtracts the block's contribution
// from the rest, so a solve costs 2 ceil(n/16) CTA barriers.  x_j = y_j * (1 / R_jj) with the
// reciprocals computed once per factorisation; that perturbs each diagonal
// entry by at most two roundings, so the solve stays backward stable.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kTB = 16;  // diagonal block size
static_assert(LSQ_MAX_N <= kVecThreads, "block_trsv takes one thread per row");

// Entry (jj, l) of the diagonal block starting at j0 (len = its size): column
// j0+jj of R for R x = y, row j0+jj for R^T x = y; 0 outside the block.
__device__ __forceinline__ double diag_entry(const double *__restrict__ Rb, int n, int j0, int len,
                                             int e) {
  const int jj = e / kTB, l = e % kTB;
  return (jj < len && l < len) ? Rb[(size_t)(j0 + jj) * n + j0 + l] : 0.0;
}

// Solve R x = y (trans 0, blocks last to first) or R^T x = y (trans 1) in
// place on sy (n doubles of shared memory).  tile: 2 kTB (kTB + 1) doubles of
// shared memory.  One thread per row (n <= blockDim.x).  Each round issues
// the loads it will need next -- this round's kTB entries of R per row and
// the next diagonal block -- before warp 0 runs the block's serial chain, so
// their L2 latency overlaps the chain instead of following it.
__device__ void block_trsv(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                           const double *__restrict__ rinv, int n, int trans, double *sy,
                           double *tile) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (n + kTB - 1) / kTB;
  const double *Rb = trans ? Rrm : Rcm;
  constexpr int TS = kTB * (kTB + 1);
  {
    const int blk = trans ? 0 : nb - 1, j0 = blk * kTB, len = min(n, j0 + kTB) - j0;
    if (tid < kTB * kTB) tile[(tid / kTB) * (kTB + 1) + tid % kTB] = diag_entry(Rb, n, j0, len, tid);
  }
  __syncthreads();
  for (int bb = 0; bb < nb; bb++) {
    const int blk = trans ? bb : nb - 1 - bb;
    const int j0 = blk * kTB, j1 = min(n, j0 + kTB), len = j1 - j0;
    const double *tcur = tile + (bb & 1) * TS;
    double *tnext = tile + ((bb + 1) & 1) * TS;
    double tv = 0.0;
    if (bb + 1 < nb && tid < kTB * kTB) {
      const int nblk = trans ? bb + 1 : nb - 2 - bb, nj0 = nblk * kTB;
      tv = diag_entry(Rb, n, nj0, min(n, nj0 + kTB) - nj0, tid);
    }
    const int ib = trans ? j1 : 0, ie = trans ? n : j0;
    const int i = ib + tid;
    const bool upd = i < ie;
    double rv[kTB];
#pragma unroll
    for (int jj = 0; jj < kTB; jj++)
      rv[jj] = (upd && jj < len) ? Rb[(size_t)(j0 + jj) * n + i] : 0.0;
    if (warp == 0) {
      double yl = (lane < len) ? sy[j0 + lane] : 0.0;
      const double ri = (lane < len) ? rinv[j0 + lane] : 0.0;
      if (!trans) {
        for (int jj = len - 1; jj >= 0; jj--) {
          const double xj = __shfl_sync(0xffffffffu, yl * ri, jj);
          if (lane == jj) yl = xj;
          else if (lane < jj) yl = fma(-tcur[jj * (kTB + 1) + lane], xj, yl);
        }
      } else {
        for (int jj = 0; jj < len; jj++) {
          const double xj = __shfl_sync(0xffffffffu, yl * ri, jj);
          if (lane == jj) yl = xj;
          else if (lane > jj && lane < len) yl = fma(-tcur[jj * (kTB + 1) + lane], xj, yl);
        }
      }
      if (lane < len) sy[j0 + lane] = yl;
    }
    __syncthreads();
    // subtract the block's contribution from the remaining rows; four
    // independent accumulators keep the FP64 FMA chains short
    if (upd) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
      for (int jj = 0; jj < kTB; jj += 4) {
        a0 = fma(rv[jj], (jj < len) ? sy[j0 + jj] : 0.0, a0);
        a1 = fma(rv[jj + 1], (jj + 1 < len) ? sy[j0 + jj + 1] : 0.0, a1);
        a2 = fma(rv[jj + 2], (jj + 2 < len) ? sy[j0 + jj + 2] : 0.0, a2);
        a3 = fma(rv[jj + 3], (jj + 3 < len) ? sy[j0 + jj + 3] : 0.0, a3);
      }
      sy[i] -= (a0 + a1) + (a2 + a3);
    }
    if (bb + 1 < nb && tid < kTB * kTB) tnext[(tid / kTB) * (kTB + 1) + tid % kTB] = tv;
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

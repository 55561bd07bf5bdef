// Triangular solves with the preconditioner R by back substitution (the
// analysis computes every R^{-1} z and R^{-T} z this way: Sec. 6, notation,
// and Proposition 6.5), and the condest / normest estimates of R that the
// step-1 stopping rule and the q0 count use (Sec. 4.2; Alg. 4 reads them off
// the SVD of SA, whose singular values equal those of R).
//
// One CTA per solve: the vector lives in shared memory; R (n x n) is read
// from L2 in both layouts so that every access is coalesced -- column j of R
// (column-major copy) for R x = y, row j of R (row-major copy) for R^T x = y.
// Blocked by 32: warp 0 solves each 32 x 32 diagonal block with shuffles
// while other warps subtract the previous block's contribution from the
// remaining rows (see block_trsv).  x_j = y_j * (1 / R_jj) with the
// reciprocals computed once per factorisation; that perturbs each diagonal
// entry by at most two roundings, so the solve stays backward stable.
#include "lsq_common.cuh"
#include "lsq_cluster.cuh"

namespace lsq {

namespace {

static_assert(kVecThreads == 1024, "block_trsv's warp roles assume 32 warps");
static_assert(LSQ_MAX_N <= 24 * 32 * 2, "bulk warps take at most two rows per round");

constexpr int kSolveThreads = 32 + 24 * 32;  // the solver warp and the 24 bulk warps
constexpr int kTile = 32 * 33;               // one 32 x 32 tile, padded rows

__device__ __forceinline__ void bar_arrive(int id) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(kSolveThreads) : "memory");
}
__device__ __forceinline__ void bar_wait(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kSolveThreads) : "memory");
}
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Warp-level asynchronous copy of a 32 x 32 tile into shared memory:
// dst[jj * 33 + l] = src[(c0 + jj) * ld + r0 + l] for jj < ncol, l < nrow, else 0.
__device__ __forceinline__ void tile_async(double *dst, const double *__restrict__ src, int ld,
                                           int c0, int ncol, int r0, int nrow, int lane) {
  for (int jj = 0; jj < 32; jj++) {
    if (jj < ncol && lane < nrow) cp_async8(dst + jj * 33 + lane, src + (size_t)(c0 + jj) * ld + r0 + lane);
    else dst[jj * 33 + lane] = 0.0;
  }
}

// Solve R x = y (trans 0; blocks last to first) or R^T x = y (trans 1; first
// to last) in place on sy (n doubles of shared memory); tile: 3 kTile
// doubles of shared memory.  Blocks of 32.  Roles (1024 threads):
//   * warp 0, the solver: for each block, the serial chain on the diagonal
//     tile, then the "lookahead" update of the next block's rows with the
//     block's x.  The diagonal and off-diagonal tiles it needs next are
//     fetched with asynchronous copies while it works.
//   * 24 bulk warps (warp % 4 != 0, so none shares warp 0's scheduler): the
//     update of every row beyond the next block with the block's x.
//   * the other 7 warps wait at the final barrier.
// The solver hands x of round r to the bulk warps with a named barrier
// (bar.arrive / bar.sync), and before its lookahead of round r waits for
// the bulk update of round r-1 (the same rows).  Rounds alternate between
// two barrier ids per direction, so an arrival for round r+2 can never fall
// into round r's barrier.  The solver's chain therefore overlaps the bulk
// update, whose FP64 work sets the pace only in the first rounds.
__device__ void block_trsv(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                           const double *__restrict__ rinv, const double *__restrict__ Dt, int n,
                           int trans, double *sy, double *tile) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (n + 31) / 32;
  const double *Rb = trans ? Rrm : Rcm;
  const double *Db = Dt + (size_t)trans * nb * 1024;  // this direction's scaled diagonal blocks
  double *otile = tile + 2 * kTile;
  if (warp == 0) {
    const int blk0 = trans ? 0 : nb - 1;
    tile_async(tile, Db + (size_t)blk0 * 1024, 32, 0, 32, 0, 32, lane);
    cp_async_commit();
    for (int r = 0; r < nb; r++) {
      const int blk = trans ? r : nb - 1 - r;
      const int j0 = blk * 32, len = min(n, j0 + 32) - j0;
      const bool has_next = r + 1 < nb;
      const int nblk = trans ? r + 1 : nb - 2 - r;
      const int nj0 = nblk * 32, nlen = has_next ? min(n, nj0 + 32) - nj0 : 0;
      const double *dt = tile + (r & 1) * kTile;
      __syncwarp();
      if (has_next) {
        tile_async(tile + ((r + 1) & 1) * kTile, Db + (size_t)nblk * 1024, 32, 0, 32, 0, 32, lane);
        tile_async(otile, Rb, n, j0, len, nj0, nlen, lane);  // rows of the next block
      }
      cp_async_commit();
      cp_async_wait<1>();
      __syncwarp();
      // the block's rows scaled by 1 / R_ll: with the tile pre-scaled the
      // same way, each step of the chain is one shuffle and one FMA
      double zl = (lane < len) ? sy[j0 + lane] * rinv[j0 + lane] : 0.0;
      if (!trans) {
        for (int jj = len - 1; jj >= 0; jj--) {
          const double xj = __shfl_sync(0xffffffffu, zl, jj);
          if (lane < jj) zl = fma(-dt[jj * 33 + lane], xj, zl);
        }
      } else {
        for (int jj = 0; jj < len; jj++) {
          const double xj = __shfl_sync(0xffffffffu, zl, jj);
          if (lane > jj && lane < len) zl = fma(-dt[jj * 33 + lane], xj, zl);
        }
      }
      if (lane < len) sy[j0 + lane] = zl;
      __syncwarp();
      bar_arrive(1 + (r & 1));              // x of this block is in sy
      if (r >= 1) bar_wait(3 + ((r - 1) & 1));  // bulk update of round r-1 done
      if (has_next) {
        cp_async_wait<0>();
        __syncwarp();
        if (lane < nlen) {
          double a0 = 0.0, a1 = 0.0;
          for (int jj = 0; jj + 1 < len; jj += 2) {
            a0 = fma(otile[jj * 33 + lane], sy[j0 + jj], a0);
            a1 = fma(otile[(jj + 1) * 33 + lane], sy[j0 + jj + 1], a1);
          }
          if (len & 1) a0 = fma(otile[(len - 1) * 33 + lane], sy[j0 + len - 1], a0);
          sy[nj0 + lane] -= a0 + a1;
        }
      }
    }
    bar_wait(3 + ((nb - 1) & 1));  // the bulk warps' last round
  } else if (warp & 3) {
    const int bt = (warp - 1 - (warp >> 2)) * 32 + lane;  // 0 .. 767
    for (int r = 0; r < nb; r++) {
      const int blk = trans ? r : nb - 1 - r;
      const int j0 = blk * 32, j1 = min(n, j0 + 32), len = j1 - j0;
      // rows beyond the next block
      const int lo = trans ? min(n, j1 + 32) : 0, hi = trans ? n : max(0, j0 - 32);
      bar_wait(1 + (r & 1));
      for (int i = lo + bt; i < hi; i += 24 * 32) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int jj = 0;
        for (; jj + 3 < len; jj += 4) {
          a0 = fma(Rb[(size_t)(j0 + jj) * n + i], sy[j0 + jj], a0);
          a1 = fma(Rb[(size_t)(j0 + jj + 1) * n + i], sy[j0 + jj + 1], a1);
          a2 = fma(Rb[(size_t)(j0 + jj + 2) * n + i], sy[j0 + jj + 2], a2);
          a3 = fma(Rb[(size_t)(j0 + jj + 3) * n + i], sy[j0 + jj + 3], a3);
        }
        for (; jj < len; jj++) a0 = fma(Rb[(size_t)(j0 + jj) * n + i], sy[j0 + jj], a0);
        sy[i] -= (a0 + a1) + (a2 + a3);
      }
      bar_arrive(3 + (r & 1));
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kVecThreads)
    trsv_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                const double *__restrict__ rinv, const double *__restrict__ Dt, int n, int trans,
                const double *y,
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
  block_trsv(Rcm, Rrm, rinv, Dt, n, trans, sy, tile);
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
__device__ void condest_body(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                             const double *__restrict__ rinv, const double *__restrict__ Dt, int n,
                             int iters, DevState *st, double *sm) {
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
    block_trsv(Rcm, Rrm, rinv, Dt, n, 1, v, tile);  // v <- R^{-T} v
    winv = block_normalize(v, n, scratch);
    if (it == iters) break;
    block_trsv(Rcm, Rrm, rinv, Dt, n, 0, v, tile);  // v <- R^{-1} v
    block_normalize(v, n, scratch);
  }
  if (threadIdx.x == 0) {
    const double smin = (winv > 0.0) ? 1.0 / winv : 0.0;
    st->normest = smax;
    st->condest = (smin > 0.0) ? smax / smin : INFINITY;
  }
}

__global__ void __launch_bounds__(kVecThreads)
    condest_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                   const double *__restrict__ rinv, const double *__restrict__ Dt, int n, int iters,
                   DevState *st) {
  extern __shared__ double sm[];
  condest_body(Rcm, Rrm, rinv, Dt, n, iters, st, sm);
}

// ---------------------------------------------------------------------------
// Batched forms (one CTA of kVecThreads per item, lsq_batch.cu).
// ---------------------------------------------------------------------------

// Step-2 count: q0 of Theorem 7.1 with kappa := condest and distortion
// 1.01 eta; Alg. 5 returns dy_(q) after q - 1 updates (as the plan path).
__device__ int step2_count(double condest, double eta, int max_inner) {
  const double e = 1.01 * eta;
  double q0 = 11.0;
  if (e > 0.0 && isfinite(condest) && condest > 0.0) {
    const double v = 1.0 + 2.0 * log(1.0 / (condest * kU)) / log(1.0 / e);
    q0 = v > 11.0 ? v : 11.0;
  }
  int q = (int)ceil(q0) - 1;
  if (q < 1) q = 1;
  if (q > max_inner) q = max_inner;
  return q;
}

// After the QR: R (both layouts), 1/R_ii, t, the scaled diagonal tiles,
// condest / normest, x0 = R^-1 t (xs; xo = D^-1 xs; ||x0||^2) and q2.
__global__ void __launch_bounds__(kVecThreads)
    b_setup_kernel(const BItem *__restrict__ items, int iters, int max_inner) {
  extern __shared__ double sm[];
  const BItem &it = items[blockIdx.x];
  const int n = it.n, d = it.d, nb = (n + 31) / 32;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int j = idx / n, i = idx % n;  // column j, row i
    const double v = (i <= j) ? it.W[(size_t)j * d + i] : 0.0;
    it.Rcm[(size_t)j * n + i] = v;
    it.Rrm[(size_t)i * n + j] = v;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    it.rinv[i] = 1.0 / it.W[(size_t)i * d + i];
    it.t[i] = it.W[(size_t)n * d + i];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * nb * 1024; idx += blockDim.x) {
    const int blk = idx / 1024, e = idx % 1024, tr = blk / nb, b = blk % nb;
    const int jj = e >> 5, l = e & 31, j0 = b * 32, len = min(n, j0 + 32) - j0;
    const double *Rb = tr ? it.Rrm : it.Rcm;
    it.Dt[idx] = (jj < len && l < len) ? Rb[(size_t)(j0 + jj) * n + j0 + l] * it.rinv[j0 + l] : 0.0;
  }
  __syncthreads();
  condest_body(it.Rcm, it.Rrm, it.rinv, it.Dt, n, iters, it.st, sm);
  __syncthreads();
  double *sy = sm, *scratch = sm + n, *tile = scratch + 32;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sy[i] = it.t[i];
  __syncthreads();
  block_trsv(it.Rcm, it.Rrm, it.rinv, it.Dt, n, 0, sy, tile);
  double nrm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    it.xs[i] = sy[i];
    it.xo[i] = it.dinv[i] * sy[i];
    nrm = fma(sy[i], sy[i], nrm);
  }
  nrm = block_sum(nrm, scratch);
  if (threadIdx.x == 0) {
    it.st->x0norm2 = nrm;
    it.st->q2 = step2_count(it.st->condest, it.eta, max_inner);
    it.st->alpha = it.alpha;
    it.st->beta = it.beta;
  }
}

// The triangular solves of the refinement loop for every item (see
// launch_b_trsv for the modes).
__global__ void __launch_bounds__(kVecThreads)
    b_trsv_kernel(const BItem *__restrict__ items, int mode, int step) {
  const BItem &it = items[blockIdx.x];
  if (mode <= 1 && *(volatile const int *)&it.st->done) return;
  extern __shared__ double sm[];
  const int n = it.n;
  double *sy = sm, *scratch = sm + n, *tile = scratch + 32;
  const double *src = mode == 0 ? (it.method == 0 ? it.dy : it.p)
                      : mode == 1 ? it.h : mode == 2 ? it.g : it.dy;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sy[i] = src[i];
  __syncthreads();
  block_trsv(it.Rcm, it.Rrm, it.rinv, it.Dt, n, (mode == 1 || mode == 2) ? 1 : 0, sy, tile);
  double nrm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = sy[i];
    if (mode == 0) {
      it.z[i] = it.dinv[i] * x;
    } else if (mode == 1) {
      it.w[i] = x;
    } else if (mode == 2) {
      it.c[i] = x;
      nrm = fma(x, x, nrm);
    } else {
      const double xs = it.xs[i] + x;
      it.xs[i] = xs;
      it.xo[i] = it.dinv[i] * xs;
    }
  }
  if (mode == 2) {
    nrm = block_sum(nrm, scratch);
    if (threadIdx.x == 0) it.st->cnorm2[step] = nrm;
  }
}

// ---------------------------------------------------------------------------
// Cluster form of the substitution for one vector.  GB300 issues one FP64
// warp instruction per 64 cycles per SM sub-partition (1.7 FMA per clock per
// SM), so one CTA spends most of a solve on the n^2 / 2 updates of the rows
// beyond the next block.  Here a cluster of kClusterCtas CTAs shares it:
//   * CTA 0, the chain CTA: warp 0 solves each 32 x 32 diagonal block (one
//     shuffle and one FMA per step, the tiles pre-scaled by 1 / R_ll);
//     warps 1-3 (the other sub-partitions) apply the block's x to the next
//     block's rows (the lookahead), a third of the columns each;
//   * CTAs 1..7, the update CTAs: block k belongs to CTA 1 + k % 7, one warp
//     per block with its running sums in registers.  Each x block that CTA 0
//     broadcasts is applied to the owned blocks beyond the next one; once a
//     block has its last such update (two rounds before it is solved) its
//     sums go to CTA 0.
// x travels CTA 0 -> CTAs 1..7 and the sums CTAs 1..7 -> CTA 0 by st.async
// into the receiver's shared memory, each transfer completing an mbarrier of
// the receiver that is used once.  The chain thus waits only on its own work
// and on sums that were sent a round earlier.  Each inner product still runs
// over the same terms, so the solve is backward stable as before.  Every
// wait is bounded; a timeout records LSQ_ERR_TIMEOUT in *err.
// ---------------------------------------------------------------------------
constexpr int kClusterCtas = 8;
constexpr int kClusterMinN = 97;  // four or more blocks: below, one CTA does as well
constexpr int kUpdateCtas = kClusterCtas - 1;
constexpr int kClusterThreads = 256;
constexpr int kMaxBlocks = (LSQ_MAX_N + 31) / 32;
constexpr uint64_t kClusterWaitNs = 1000ull * 1000 * 1000;  // 1 s
static_assert(kMaxBlocks <= kUpdateCtas * (kClusterThreads / 32), "one warp per owned block");

__device__ bool xfer_wait(uint64_t *bar) { return xfer_wait_limit(bar, kClusterWaitNs); }
__device__ __forceinline__ void nbar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nbar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
// Round r solves block blk_of(r); the map is its own inverse (block k is
// solved in round blk_of(k)).
__device__ __forceinline__ int blk_of(int r, int nb, int trans) { return trans ? r : nb - 1 - r; }
__device__ __forceinline__ int blk_len(int k, int n) { return min(n, 32 * k + 32) - 32 * k; }
// the last round whose x update CTA `rank` (1..7) applies, plus 2
__device__ __forceinline__ int update_last(int rank, int nb, int trans) {
  int mp = -1;
  for (int k = rank - 1; k < nb; k += kUpdateCtas) mp = max(mp, blk_of(k, nb, trans));
  return mp;
}

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
    trsv_cluster_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                        const double *__restrict__ rinv, const double *__restrict__ Dt, int n,
                        int trans, const double *y, const double *in_scale, double *out,
                        const double *out_scale, double *out_scaled, double *accum,
                        double *norm2_out, const DevState *gate, int *err) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  const int rank = (int)cluster_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (n + 31) / 32;
  const double *Rb = trans ? Rrm : Rcm;
  // shared: sx (x of the solved blocks, padded to 32 nb), ps (CTA 0: the
  // shipped sums), lp (CTA 0: lookahead partials of warps 1-3), scratch,
  // then one transfer mbarrier per block (CTA 0) or per round (CTAs 1..7)
  extern __shared__ __align__(16) double csm[];
  double *sx = csm, *ps = csm + 32 * nb, *lp = ps + 32 * nb, *scratch = lp + 96;
  uint64_t *bars = reinterpret_cast<uint64_t *>(scratch + 8);
  for (int i = threadIdx.x; i < 32 * nb; i += blockDim.x) sx[i] = ps[i] = 0.0;
  const int last = rank == 0 ? 0 : update_last(rank, nb, trans);
  if (threadIdx.x == 0) {
    if (rank == 0) {
      for (int k = 0; k < nb; k++)
        if (blk_of(k, nb, trans) >= 2) xfer_bar_init(bars + k, 8u * blk_len(k, n));
    } else {
      for (int r = 0; r <= last - 2; r++) xfer_bar_init(bars + r, 8u * blk_len(blk_of(r, nb, trans), n));
    }
    fence_mbarrier_init_cluster();
  }
  __syncthreads();
  cluster_sync_all();  // every barrier is armed before any remote store
  bool ok = true;
  if (rank == 0 && warp == 0) {
    // the last round + 2 of update CTA lane + 1, for the broadcast
    const int lastl = lane < kUpdateCtas ? update_last(lane + 1, nb, trans) : -1;
    double dreg[32], rl = 0.0;  // the block's scaled diagonal tile and 1 / R_ll
    auto load_diag = [&](int k) {
      const double *D = Dt + ((size_t)trans * nb + k) * 1024;
#pragma unroll
      for (int jj = 0; jj < 32; jj++) dreg[jj] = D[jj * 32 + lane];
      rl = lane < blk_len(k, n) ? rinv[32 * k + lane] : 0.0;
    };
    load_diag(blk_of(0, nb, trans));
    for (int r = 0; r < nb; r++) {
      const int l = blk_of(r, nb, trans), j0 = 32 * l, len = blk_len(l, n);
      double zb;
      if (r < 2) {
        zb = (lane < len) ? (in_scale ? y[j0 + lane] * in_scale[j0 + lane] : y[j0 + lane]) : 0.0;
      } else {
        if (!xfer_wait(bars + l)) ok = false;
        zb = ps[j0 + lane];
      }
      if (r >= 1) {
        nbar_sync(3 + (r & 1), 128);  // lookahead of round r - 1 on this block
        zb -= (lp[lane] + lp[32 + lane]) + lp[64 + lane];
      }
      double zl = zb * rl;
      if (!trans) {
#pragma unroll
        for (int jj = 31; jj >= 0; jj--) {
          if (jj < len) {
            const double xj = __shfl_sync(0xffffffffu, zl, jj);
            if (lane < jj) zl = fma(-dreg[jj], xj, zl);
          }
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < 32; jj++) {
          if (jj < len) {
            const double xj = __shfl_sync(0xffffffffu, zl, jj);
            if (lane > jj && lane < len) zl = fma(-dreg[jj], xj, zl);
          }
        }
      }
      if (lane < len) sx[j0 + lane] = zl;
      __syncwarp();
      if (r + 1 < nb) {
        nbar_arrive(1 + (r & 1), 128);  // x of round r for the lookahead warps
        load_diag(blk_of(r + 1, nb, trans));
      }
      for (int b = 1; b <= kUpdateCtas; b++) {
        const int lb = __shfl_sync(0xffffffffu, lastl, b - 1);
        if (lb >= r + 2 && lane < len)
          st_async_f64(cluster_addr(sx + j0 + lane, b), zl, cluster_addr(bars + r, b));
      }
    }
  } else if (rank == 0 && warp <= 3) {
    // lookahead: columns [c0, c0 + 11) of the solved block on the next block's rows
    const int c0 = 11 * (warp - 1);
    for (int r = 0; r + 1 < nb; r++) {
      const int l = blk_of(r, nb, trans), j0 = 32 * l, len = blk_len(l, n);
      const int ln = blk_of(r + 1, nb, trans), i = 32 * ln + lane, lenn = blk_len(ln, n);
      double rv[11];
#pragma unroll
      for (int q = 0; q < 11; q++) {
        const int jj = c0 + q;
        rv[q] = (jj < 32 && jj < len && lane < lenn) ? Rb[(size_t)(j0 + jj) * n + i] : 0.0;
      }
      nbar_sync(1 + (r & 1), 128);
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int q = 0; q < 11; q++) {
        const int jj = c0 + q;
        const double xv = jj < 32 ? sx[j0 + jj] : 0.0;
        if (q & 1) a1 = fma(rv[q], xv, a1);
        else a0 = fma(rv[q], xv, a0);
      }
      lp[32 * (warp - 1) + lane] = a0 + a1;
      nbar_arrive(3 + ((r + 1) & 1), 128);
    }
  } else if (rank > 0) {
    const int k = rank - 1 + kUpdateCtas * warp;  // this warp's block
    if (k < nb && blk_of(k, nb, trans) >= 2) {
      const int pk = blk_of(k, nb, trans), i0 = 32 * k, lenk = blk_len(k, n), i = i0 + lane;
      double S = (lane < lenk) ? (in_scale ? y[i] * in_scale[i] : y[i]) : 0.0;
      for (int r = 0; r <= pk - 2; r++) {
        const int l = blk_of(r, nb, trans), j0 = 32 * l, len = blk_len(l, n);
        double rv[32];  // R does not depend on x: loaded before the wait
#pragma unroll
        for (int jj = 0; jj < 32; jj++)
          rv[jj] = (jj < len && lane < lenk) ? Rb[(size_t)(j0 + jj) * n + i] : 0.0;
        if (!xfer_wait(bars + r)) ok = false;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int jj = 0; jj < 32; jj += 4) {
          a0 = fma(rv[jj], sx[j0 + jj], a0);
          a1 = fma(rv[jj + 1], sx[j0 + jj + 1], a1);
          a2 = fma(rv[jj + 2], sx[j0 + jj + 2], a2);
          a3 = fma(rv[jj + 3], sx[j0 + jj + 3], a3);
        }
        S -= (a0 + a1) + (a2 + a3);
      }
      if (lane < lenk) st_async_f64(cluster_addr(ps + i0 + lane, 0), S, cluster_addr(bars + k, 0));
    }
  }
  if (!ok) {
    if (err != nullptr) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
    // let late transfers into this CTA land before it exits (bounded)
    if (rank == 0) {
      for (int k = 0; k < nb; k++)
        if (blk_of(k, nb, trans) >= 2) xfer_wait(bars + k);
    } else {
      for (int r = 0; r <= last - 2; r++) xfer_wait(bars + r);
    }
  }
  __syncthreads();
  if (rank == 0) {
    double nrm = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double x = sx[i];
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
  cluster_sync_all();  // no CTA leaves while another may still address it
}

// Dt[t][b][jj][l] = (t ? Rrm : Rcm)[(32b + jj) n + 32b + l] / R_(32b+l)(32b+l):
// block b's diagonal tile for R x = y (t = 0) or R^T x = y (t = 1), each
// entry scaled by the reciprocal diagonal of the row it updates; zero
// outside the block.  One CTA of 1024 threads per (t, b).
__global__ void __launch_bounds__(1024)
    diag_tiles_kernel(const double *__restrict__ Rcm, const double *__restrict__ Rrm,
                      const double *__restrict__ rinv, int n, double *Dt) {
  const int nb = (n + 31) / 32;
  const int t = blockIdx.x / nb, b = blockIdx.x % nb;
  const int jj = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int j0 = b * 32, len = min(n, j0 + 32) - j0;
  const double *Rb = t ? Rrm : Rcm;
  Dt[(size_t)blockIdx.x * 1024 + threadIdx.x] =
      (jj < len && l < len) ? Rb[(size_t)(j0 + jj) * n + j0 + l] * rinv[j0 + l] : 0.0;
}

}  // namespace

cudaError_t launch_diag_tiles(const double *Rcm, const double *Rrm, const double *rinv, int n,
                              double *Dt, cudaStream_t s) {
  diag_tiles_kernel<<<2 * ((n + 31) / 32), 1024, 0, s>>>(Rcm, Rrm, rinv, n, Dt);
  return cudaGetLastError();
}

cudaError_t launch_trsv(const double *Rcm, const double *Rrm, const double *rinv, const double *Dt,
                        int n, int trans,
                        const double *y, const double *in_scale, double *out,
                        const double *out_scale, double *out_scaled, double *accum,
                        double *norm2_out, const DevState *gate, cudaStream_t s, int batch,
                        int64_t bstride, int *err) {
  if (batch == 1 && n >= kClusterMinN) {
    const int nb = (n + 31) / 32;
    const size_t csmem = (size_t)(64 * nb + 96 + 8) * sizeof(double) + sizeof(uint64_t) * nb;
    trsv_cluster_kernel<<<kClusterCtas, kClusterThreads, csmem, s>>>(
        Rcm, Rrm, rinv, Dt, n, trans, y, in_scale, out, out_scale, out_scaled, accum, norm2_out,
        gate, err);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)(n + 32 + 3 * kTile) * sizeof(double);
  trsv_kernel<<<batch, kVecThreads, smem, s>>>(Rcm, Rrm, rinv, Dt, n, trans, y, in_scale, out,
                                               out_scale, out_scaled, accum, norm2_out, gate,
                                               bstride);
  return cudaGetLastError();
}

cudaError_t prepare_b_kernels(int nmax) {
  const size_t smem = (size_t)(2 * nmax + 32 + 3 * kTile) * sizeof(double);
  cudaError_t e = ensure_smem_attr((const void *)b_setup_kernel, (int)smem);
  if (e == cudaSuccess) e = ensure_smem_attr((const void *)b_trsv_kernel, (int)smem);
  return e;
}

cudaError_t launch_b_setup(const BItem *items, int count, int cond_iters, int max_inner,
                           int nmax, cudaStream_t s) {
  const size_t smem = (size_t)(2 * nmax + 32 + 3 * kTile) * sizeof(double);
  cudaError_t e = ensure_smem_attr((const void *)b_setup_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  b_setup_kernel<<<count, kVecThreads, smem, s>>>(items, cond_iters, max_inner);
  return cudaGetLastError();
}

cudaError_t launch_b_trsv(const BItem *items, int count, int mode, int step, int nmax,
                          cudaStream_t s) {
  const size_t smem = (size_t)(nmax + 32 + 3 * kTile) * sizeof(double);
  cudaError_t e = ensure_smem_attr((const void *)b_trsv_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  b_trsv_kernel<<<count, kVecThreads, smem, s>>>(items, mode, step);
  return cudaGetLastError();
}

cudaError_t launch_condest(const double *Rcm, const double *Rrm, const double *rinv,
                           const double *Dt, int n, int iters, DevState *st, cudaStream_t s) {
  const size_t smem = (size_t)(2 * n + 32 + 3 * kTile) * sizeof(double);
  condest_kernel<<<1, kVecThreads, smem, s>>>(Rcm, Rrm, rinv, Dt, n, iters, st);
  return cudaGetLastError();
}

}  // namespace lsq

// Many right-hand sides on one matrix: k solves share one sketch S [A B] and
// one QR (the augmented columns carry Q^T S B), and the two passes of the
// refinement loop become dense contractions over row blocks of A:
//   resid:  G = A^T (B - A X)      inner:  H = A^T (A Z)        (Z, X: n x k)
// (Alg. 1's refinement right-hand side and Apply, column by column).
//
// GB300 design: one CTA per SM streams its contiguous rows in blocks of 32:
// the block of A (32 x n) and Z (n x k) sit in shared memory; T = A_blk Z
// (32 x k) and then H += A_blk^T T (n x k, accumulated in registers across
// all blocks) are FP64 tensor-core MMAs (mma.sync m8n8k4 .f64); the CTA
// writes one n x k partial, reduced in a fixed order.  The FP64 tensor rate
// of GB300 (about 1 TFLOP/s) makes this pass compute-bound: 4 m n k flops
// against 8 m n bytes.
//
// Limits: n <= 256 (n rounded up to 8), k a multiple of 8 and <= 64.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kMBlock = 32;       // rows of A per block
constexpr int kMultiThreads = 256;
constexpr int kMaxNp8 = 256;

__device__ __forceinline__ void dmma(double &c0, double &c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

// Fragment layout of m8n8k4 (f64): A (8x4, row) element a[lane/4][lane%4];
// B (4x8, col) element b[lane%4][lane/4]; C (8x8) elements c[lane/4][2(lane%4)+{0,1}].
template <int NT, bool RESID>
__global__ void __launch_bounds__(kMultiThreads, 1)
    multi_pass_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n, int np8,
                      const double *__restrict__ Zcm, const double *__restrict__ B, int64_t ldb,
                      double *__restrict__ part, double *__restrict__ r2part,
                      const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  constexpr int K = NT * 8;
  extern __shared__ double sm[];
  const int lsa = np8 + 1, lsz = K + 1, lst = K + 1;
  double *sA = sm;                          // kMBlock x lsa
  double *sZ = sA + kMBlock * lsa;          // np8 x lsz
  double *sT = sZ + (size_t)np8 * lsz;      // kMBlock x lst
  double *sR2 = sT + kMBlock * lst;         // K
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int fr = lane >> 2, fc = lane & 3;  // fragment row / column
  const int MT = np8 / 8;
  for (int idx = tid; idx < np8 * K; idx += blockDim.x) {
    const int j = idx / K, c = idx % K;
    sZ[j * lsz + c] = (j < n) ? Zcm[(size_t)c * n + j] : 0.0;
  }
  if (RESID)
    for (int c = tid; c < K; c += blockDim.x) sR2[c] = 0.0;
  double acc[4][NT][2];
#pragma unroll
  for (int q = 0; q < 4; q++)
#pragma unroll
    for (int t = 0; t < NT; t++) acc[q][t][0] = acc[q][t][1] = 0.0;

  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  for (int64_t rb = r0; rb < r1; rb += kMBlock) {
    __syncthreads();
    for (int idx = tid; idx < kMBlock * np8; idx += blockDim.x) {
      const int i = idx / np8, j = idx % np8;
      sA[i * lsa + j] = (rb + i < r1 && j < n) ? __ldcs(A + (rb + i) * lda + j) : 0.0;
    }
    __syncthreads();
    // phase 1: T = A_blk Z  (4 x NT tiles of 8 x 8)
    for (int t = warp; t < 4 * NT; t += kMultiThreads / 32) {
      const int mt = t & 3, nt = t >> 2;
      double c0 = 0.0, c1 = 0.0;
      for (int kk = 0; kk < np8 / 4; kk++) {
        const double a = sA[(mt * 8 + fr) * lsa + kk * 4 + fc];
        const double b = sZ[(kk * 4 + fc) * lsz + nt * 8 + fr];
        dmma(c0, c1, a, b);
      }
      const int row = mt * 8 + fr, col = nt * 8 + 2 * fc;
      if (RESID) {
        const bool ok = rb + row < r1;
        const double b0 = ok ? B[(rb + row) * ldb + col] : 0.0;
        const double b1 = ok ? B[(rb + row) * ldb + col + 1] : 0.0;
        c0 = b0 - c0;
        c1 = b1 - c1;
        if (ok) {
          atomicAdd(sR2 + col, c0 * c0);
          atomicAdd(sR2 + col + 1, c1 * c1);
        } else {
          c0 = c1 = 0.0;
        }
      }
      sT[row * lst + col] = c0;
      sT[row * lst + col + 1] = c1;
    }
    __syncthreads();
    // phase 2: H += A_blk^T T  (MT x NT tiles, K-dimension = the 32 rows)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int mt = warp + 8 * q;
      if (mt < MT) {
#pragma unroll
        for (int kk = 0; kk < kMBlock / 4; kk++) {
          const double a = sA[(kk * 4 + fc) * lsa + mt * 8 + fr];
#pragma unroll
          for (int nt = 0; nt < NT; nt++) {
            const double b = sT[(kk * 4 + fc) * lst + nt * 8 + fr];
            dmma(acc[q][nt][0], acc[q][nt][1], a, b);
          }
        }
      }
    }
  }
  // partial (column-major np8 x K) of this CTA
  double *P = part + (size_t)blockIdx.x * np8 * K;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int mt = warp + 8 * q;
    if (mt < MT) {
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        const int j = mt * 8 + fr, c = nt * 8 + 2 * fc;
        P[(size_t)c * np8 + j] = acc[q][nt][0];
        P[(size_t)(c + 1) * np8 + j] = acc[q][nt][1];
      }
    }
  }
  if (RESID) {
    __syncthreads();
    for (int c = tid; c < K; c += blockDim.x) r2part[(size_t)blockIdx.x * K + c] = sR2[c];
  }
}

// out (column-major n x k) = scale[j] * sum_g part[g]; r2[c] = sum_g r2part[g][c].
__global__ void multi_reduce_kernel(const double *__restrict__ part, int grid, int n, int np8,
                                    int k, const double *__restrict__ scale, double *out,
                                    const double *__restrict__ r2part, double *r2,
                                    const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)n * k) {
    const int c = (int)(idx / n), j = (int)(idx % n);
    double s = 0.0;
    for (int g = 0; g < grid; g++) s += part[((size_t)g * k + c) * np8 + j];
    out[idx] = scale ? scale[j] * s : s;
  }
  if (r2 != nullptr && idx < k) {
    double s = 0.0;
    for (int g = 0; g < grid; g++) s += r2part[(size_t)g * k + idx];
    r2[idx] = s;
  }
}

// Polyak update per column (one CTA per right-hand side); dn2[c] = ||Delta_c||^2.
__global__ void __launch_bounds__(kVecThreads)
    multi_polyak_kernel(int n, const double *__restrict__ C, const double *__restrict__ Wv,
                        double *DY, double *DYold, double *dn2, DevState *st) {
  if (*(volatile int *)&st->done) return;
  __shared__ double scratch[32];
  const double alpha = st->alpha, beta = st->beta;
  const size_t off = (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double y = DY[off + i];
    const double delta = alpha * (C[off + i] - Wv[off + i]) + beta * (y - DYold[off + i]);
    DYold[off + i] = y;
    DY[off + i] = y + delta;
    s = fma(delta, delta, s);
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) dn2[blockIdx.x] = s;
}

// Stop test over all columns: step 1 stops when every column's update is
// below its own threshold (Sec. 4.2 item 1 per column); any step stops at its cap.
__global__ void multi_stop_kernel(int k, const double *__restrict__ dn2,
                                  const double *__restrict__ thresh, DevState *st) {
  if (*(volatile int *)&st->done) return;
  if (threadIdx.x != 0) return;
  const int it = st->iters + 1;
  st->iters = it;
  bool stop = it >= st->max_iters;
  if (st->use_thresh) {
    bool all = true;
    for (int c = 0; c < k; c++) all = all && (sqrt(dn2[c]) <= thresh[c]);
    stop = stop || all;
  }
  if (stop) st->done = 1;
}

__global__ void multi_init_kernel(int64_t nk, const double *__restrict__ C, double *DY,
                                  double *DYold, int max_iters, int use_thresh, DevState *st) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < nk) {
    DY[idx] = C[idx];
    DYold[idx] = C[idx];
  }
  if (idx == 0) {
    st->iters = 0;
    st->max_iters = max_iters;
    st->use_thresh = use_thresh;
    st->done = (max_iters <= 0) ? 1 : 0;
  }
}

// thresh_c = u (gamma normest ||x0_c|| + rho condest ||b_c - A x0_c||)
__global__ void multi_thresh_kernel(int k, double gamma, double rho, const double *x0n2,
                                    const double *r2, double *thresh, const DevState *st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k)
    thresh[c] = kU * (gamma * st->normest * sqrt(x0n2[c]) + rho * st->condest * sqrt(r2[c]));
}

// W[:, n + c] (column-major, ld d) = zeta^{-1/2} SBb[:, c] (row-major d x (k+1)).
__global__ void sketch_b_to_w_kernel(const double *__restrict__ SBb, int d, int n, int k,
                                     double zinv, double *W, DevState *st) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)d * k) {
    const int c = (int)(idx / d), h = (int)(idx % d);
    const double v = SBb[(size_t)h * (k + 1) + c];
    if (!isfinite(v)) atomicExch(&st->nonfinite, 1);
    W[(size_t)(n + c) * d + h] = v * zinv;
  }
}

// X (row-major n x k) = Xcm (column-major n x k).
__global__ void cm_to_rm_kernel(const double *__restrict__ Xcm, int n, int k, double *X) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < (int64_t)n * k) {
    const int i = (int)(idx / k), c = (int)(idx % k);
    X[idx] = Xcm[(size_t)c * n + i];
  }
}

unsigned blocks_for(int64_t count, int th) { return (unsigned)((count + th - 1) / th); }

}  // namespace

int multi_np8(int n) { return (n + 7) / 8 * 8; }

size_t multi_pass_smem(int n, int k) {
  const int np8 = multi_np8(n);
  return ((size_t)kMBlock * (np8 + 1) + (size_t)np8 * (k + 1) + (size_t)kMBlock * (k + 1) + k) *
         sizeof(double);
}

bool multi_supported(int n, int k) {
  return multi_np8(n) <= kMaxNp8 && k >= 8 && k <= 64 && k % 8 == 0 &&
         multi_pass_smem(n, k) <= 227 * 1024;
}

template <bool RESID>
static cudaError_t multi_dispatch(const double *A, int64_t lda, int64_t m, int n, int k,
                                  const double *Z, const double *B, int64_t ldb, double *part,
                                  double *r2part, int grid, const DevState *gate,
                                  cudaStream_t s) {
  const int np8 = multi_np8(n);
  const size_t smem = multi_pass_smem(n, k);
  cudaError_t e = cudaSuccess;
#define LSQ_MULTI_CASE(NT_)                                                                  \
  case NT_: {                                                                                \
    auto fn = multi_pass_kernel<NT_, RESID>;                                                 \
    e = ensure_smem_attr((const void *)fn, (int)smem);                                       \
    if (e != cudaSuccess) return e;                                                          \
    fn<<<grid, kMultiThreads, smem, s>>>(A, lda, m, n, np8, Z, B, ldb, part, r2part, gate);   \
    break;                                                                                   \
  }
  switch (k / 8) {
    LSQ_MULTI_CASE(1)
    LSQ_MULTI_CASE(2)
    LSQ_MULTI_CASE(3)
    LSQ_MULTI_CASE(4)
    LSQ_MULTI_CASE(5)
    LSQ_MULTI_CASE(6)
    LSQ_MULTI_CASE(7)
    LSQ_MULTI_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef LSQ_MULTI_CASE
  return cudaGetLastError();
}

cudaError_t launch_multi_atax(const double *A, int64_t lda, int64_t m, int n, int k,
                              const double *Z, double *part, int grid, const DevState *gate,
                              cudaStream_t s) {
  return multi_dispatch<false>(A, lda, m, n, k, Z, nullptr, 0, part, nullptr, grid, gate, s);
}

cudaError_t launch_multi_resid(const double *A, int64_t lda, int64_t m, int n, int k,
                               const double *B, int64_t ldb, const double *X, double *part,
                               double *r2part, int grid, cudaStream_t s) {
  return multi_dispatch<true>(A, lda, m, n, k, X, B, ldb, part, r2part, grid, nullptr, s);
}

cudaError_t launch_multi_reduce(const double *part, int grid, int n, int k, const double *scale,
                                double *out, const double *r2part, double *r2,
                                const DevState *gate, cudaStream_t s) {
  const int64_t cnt = (int64_t)n * k > k ? (int64_t)n * k : k;
  multi_reduce_kernel<<<blocks_for(cnt, 128), 128, 0, s>>>(part, grid, n, multi_np8(n), k, scale,
                                                           out, r2part, r2, gate);
  return cudaGetLastError();
}

cudaError_t launch_multi_polyak(int n, int k, const double *C, const double *Wv, double *DY,
                                double *DYold, double *dn2, const double *thresh, DevState *st,
                                cudaStream_t s) {
  multi_polyak_kernel<<<k, kVecThreads, 0, s>>>(n, C, Wv, DY, DYold, dn2, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  multi_stop_kernel<<<1, 32, 0, s>>>(k, dn2, thresh, st);
  return cudaGetLastError();
}

cudaError_t launch_multi_init(int n, int k, const double *C, double *DY, double *DYold,
                              int max_iters, int use_thresh, DevState *st, cudaStream_t s) {
  const int64_t nk = (int64_t)n * k;
  multi_init_kernel<<<blocks_for(nk, 256), 256, 0, s>>>(nk, C, DY, DYold, max_iters, use_thresh,
                                                         st);
  return cudaGetLastError();
}

cudaError_t launch_multi_thresh(int k, double gamma, double rho, const double *x0n2,
                                const double *r2, double *thresh, const DevState *st,
                                cudaStream_t s) {
  multi_thresh_kernel<<<blocks_for(k, 64), 64, 0, s>>>(k, gamma, rho, x0n2, r2, thresh, st);
  return cudaGetLastError();
}

cudaError_t launch_sketch_b_to_w(const double *SBb, int d, int n, int k, int zeta, double *W,
                                 DevState *st, cudaStream_t s) {
  const int64_t cnt = (int64_t)d * k;
  sketch_b_to_w_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(SBb, d, n, k,
                                                            1.0 / sqrt((double)zeta), W, st);
  return cudaGetLastError();
}

cudaError_t launch_cm_to_rm(const double *Xcm, int n, int k, double *X, cudaStream_t s) {
  const int64_t cnt = (int64_t)n * k;
  cm_to_rm_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(Xcm, n, k, X);
  return cudaGetLastError();
}

}  // namespace lsq

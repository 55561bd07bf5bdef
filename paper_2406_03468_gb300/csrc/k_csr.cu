// Sparse A in CSR form (the paper's SuiteSparse runs, Sec. 5 "Runtime and
// iteration count": SPIR on sparse problems): row_ptr (m + 1 int64), col
// (nnz int32, distinct within a row), val (nnz FP64).  The sketch, the
// column norms and the passes over A read the nonzeros only; everything
// after the sketch (QR, triangular solves, refinement) is the dense path's.
//
// GB300 design.  A sparse row is a few hundred bytes, so a pass is bound by
// the FP64 pipe and the row reductions, not by HBM: a warp takes 4 rows at a
// time, reduces their 4 row products together by shuffles, and accumulates
// the column sums A^T v one row at a time in its own shared-memory copy of
// the n column sums (a row's column indices are distinct, so a warp's lanes
// never collide).  The CTA
// then adds its warps' copies in warp order into its partial, and the
// partials go through the dense path's fixed-order reduction: the passes are
// deterministic for a fixed grid.  The sketch scatters each nonzero into its
// zeta sketch rows with FP64 atomics in L2, as the dense path does below
// m n = 2^24 (rounding order not fixed).
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kCsrThreads = 256;
constexpr int kCsrWarps = kCsrThreads / 32;

__device__ __forceinline__ double csr_flip(double a, bool neg) {
  return __longlong_as_double(__double_as_longlong(a) ^
                              (neg ? (long long)0x8000000000000000ull : 0ll));
}

// this CTA's rows: a contiguous range of m / grid rows
__device__ __forceinline__ void csr_rows(int64_t m, int64_t &r0, int64_t &r1) {
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  r0 = min(m, (int64_t)blockIdx.x * per);
  r1 = min(m, r0 + per);
}

// part[blockIdx.x * npad + j] = sum over the warps, in warp order, of their
// column sums hs[w npad + j]
__device__ __forceinline__ void csr_flush(const double *hs, int npad, double *part) {
  __syncthreads();
  for (int j = threadIdx.x; j < npad; j += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kCsrWarps; w++) s += hs[(size_t)w * npad + j];
    part[(size_t)blockIdx.x * npad + j] = s;
  }
}

// The sketch S [A b] by scatter (each nonzero into its row's zeta sketch
// rows, with the row's signs; the 1 / sqrt(zeta) scale comes at the
// finalize, as for dense A) and the column sums of squares (partials).
__global__ void __launch_bounds__(kCsrThreads)
    csr_sketch_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                      const double *__restrict__ val, int64_t m, int n,
                      const double *__restrict__ b, int d, int zeta,
                      const int32_t *__restrict__ rows, const uint32_t *__restrict__ signbits,
                      double *__restrict__ SAb, double *__restrict__ colsq_part, int npad) {
  extern __shared__ double csm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *hw = csm + (size_t)warp * npad;
  for (int j = lane; j < npad; j += 32) hw[j] = 0.0;
  __syncwarp();
  const int ldsa = n + 1;
  int64_t r0, r1;
  csr_rows(m, r0, r1);
  for (int64_t i = r0 + warp; i < r1; i += kCsrWarps) {
    const int32_t *hr = rows + i * zeta;  // the row's zeta sketch rows (same for every lane)
    const uint32_t sb = signbits[i];
    if (b != nullptr && lane < zeta) {
      const int h = hr[lane];
      if ((unsigned)h < (unsigned)d)
        atomicAdd(SAb + (size_t)h * ldsa + n, csr_flip(b[i], (sb >> lane) & 1u));
    }
    const int64_t beg = rp[i], end = rp[i + 1];
    for (int64_t p = beg + lane; p < end; p += 32) {
      const int j = col[p];
      const double a = val[p];
      hw[j] = fma(a, a, hw[j]);
      for (int t = 0; t < zeta; t++) {
        const int h = __ldg(hr + t);
        if ((unsigned)h < (unsigned)d)
          atomicAdd(SAb + (size_t)h * ldsa + j, csr_flip(a, (sb >> t) & 1u));
      }
    }
    __syncwarp();
  }
  csr_flush(csm, npad, colsq_part);
}

// The row products of 4 rows reduced together: lane L holds partials v[0..3]
// of rows 0..3; after the exchange across 16 lanes (2 adds), across 8 lanes
// (1 add) and three butterfly levels (3 adds) lane L holds the full sum of
// row 2 (L >> 4) + ((L >> 3) & 1): 6 FP64 adds for 4 rows instead of 20
// (GB300 issues one FP64 warp instruction per 64 cycles per sub-partition).
// The tree is fixed, so the sums are deterministic.
__device__ __forceinline__ double reduce4(const double (&v)[4], int lane) {
  const bool h16 = lane >= 16, h8 = (lane & 8) != 0;
  const double s0 = h16 ? v[0] : v[2], s1 = h16 ? v[1] : v[3];
  const double k0 = h16 ? v[2] : v[0], k1 = h16 ? v[3] : v[1];
  const double w0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
  const double w1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
  double u = (h8 ? w1 : w0) + __shfl_xor_sync(0xffffffffu, h8 ? w0 : w1, 8);
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
  return u;
}

// One pass over the rows.  MODE 0 (inner pass): v_i = a_i . x.  MODE 1
// (residual pass): v_i = bs b_i - a_i . x with bs = *bscale (1 when NULL),
// written to rout[i] when rout != NULL, and ||v||^2 partials into r2_part.
// Both: the column sums sum_i a_i v_i into part[blockIdx.x].  A warp takes
// 4 consecutive rows at a time: their row products together (reduce4), then
// each row's column sums with the whole warp.  gate: skip the launch once
// gate->done is set (the inner loop's stop).
template <int MODE>
__global__ void __launch_bounds__(kCsrThreads)
    csr_pass_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                    const double *__restrict__ val, int64_t m, const double *__restrict__ b,
                    const double *__restrict__ x, double *__restrict__ part,
                    double *__restrict__ r2_part, int npad, const DevState *gate,
                    const double *bscale, double *rout) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  extern __shared__ double csm[];
  __shared__ double r2w[kCsrWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *hw = csm + (size_t)warp * npad;
  for (int j = lane; j < npad; j += 32) hw[j] = 0.0;
  __syncwarp();
  const double bs = (MODE == 1 && bscale != nullptr) ? *bscale : 1.0;
  double r2 = 0.0;
  int64_t r0, r1;
  csr_rows(m, r0, r1);
  for (int64_t i0 = r0 + 4 * warp; i0 < r1; i0 += 4 * kCsrWarps) {
    int64_t beg[4], end[4];
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const bool in = i0 + q < r1;
      beg[q] = in ? rp[i0 + q] : 0;
      end[q] = in ? rp[i0 + q + 1] : 0;
      double t = 0.0;
      for (int64_t p = beg[q] + lane; p < end[q]; p += 32) t = fma(val[p], __ldg(x + col[p]), t);
      v[q] = t;
    }
    const double u = reduce4(v, lane);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (i0 + q >= r1) break;
      const double t = __shfl_sync(0xffffffffu, u, ((q & 2) ? 16 : 0) + ((q & 1) ? 8 : 0));
      double c = t;
      if (MODE == 1) {
        c = (bscale != nullptr ? bs * b[i0 + q] : b[i0 + q]) - t;
        r2 = fma(c, c, r2);
        if (rout != nullptr && lane == 0) rout[i0 + q] = c;
      }
      for (int64_t p = beg[q] + lane; p < end[q]; p += 32) {
        const int j = col[p];
        hw[j] = fma(val[p], c, hw[j]);
      }
      __syncwarp();
    }
  }
  if (MODE == 1 && lane == 0) r2w[warp] = r2;
  csr_flush(csm, npad, part);
  if (MODE == 1 && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kCsrWarps; w++) s += r2w[w];
    r2_part[blockIdx.x] = s;
  }
}

// NaN / Inf among the nnz values or in b (st->nonfinite), and a structure
// that is not CSR of an m x n matrix with nnz entries (st->err =
// LSQ_ERR_INVALID): row_ptr[0] != 0, row_ptr[m] != nnz, a decreasing
// row_ptr, or a column index outside [0, n).  Reads col and val only below
// the caller's nnz.
__global__ void csr_check_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                 const double *__restrict__ val, int64_t m, int n, int64_t nnz,
                                 const double *__restrict__ b, DevState *st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false, badidx = false;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[m] != nnz)) badidx = true;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += stride) {
    if (!isfinite(val[p])) bad = true;
    if ((unsigned)col[p] >= (unsigned)n) badidx = true;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    if (!isfinite(b[i])) bad = true;
    if (rp[i + 1] < rp[i] || rp[i] < 0) badidx = true;
  }
  if (bad) atomicExch(&st->nonfinite, 1);
  if (badidx) atomicCAS(&st->err, 0, (int)LSQ_ERR_INVALID);
}

size_t csr_smem(int npad) { return sizeof(double) * (size_t)kCsrWarps * npad; }

}  // namespace

cudaError_t launch_csr_check(const int64_t *rp, const int32_t *col, const double *val, int64_t m,
                             int n, int64_t nnz, const double *b, DevState *st, int nsm,
                             cudaStream_t s) {
  csr_check_kernel<<<nsm * 4, 256, 0, s>>>(rp, col, val, m, n, nnz, b, st);
  return cudaGetLastError();
}

cudaError_t launch_csr_sketch(const int64_t *rp, const int32_t *col, const double *val, int64_t m,
                              int n, const double *b, int d, int zeta, const int32_t *rows,
                              const uint32_t *signbits, double *SAb, double *colsq_part, int grid,
                              int npad, cudaStream_t s) {
  const int smem = (int)csr_smem(npad);
  cudaError_t e = ensure_smem_attr((const void *)csr_sketch_kernel, smem);
  if (e != cudaSuccess) return e;
  csr_sketch_kernel<<<grid, kCsrThreads, smem, s>>>(rp, col, val, m, n, b, d, zeta, rows, signbits,
                                                    SAb, colsq_part, npad);
  return cudaGetLastError();
}

cudaError_t launch_csr_pass(int mode, const int64_t *rp, const int32_t *col, const double *val,
                            int64_t m, const double *b, const double *x, double *part,
                            double *r2_part, int grid, int npad, const DevState *gate,
                            const double *bscale, double *rout, cudaStream_t s) {
  const int smem = (int)csr_smem(npad);
  const void *fn = mode == 0 ? (const void *)csr_pass_kernel<0> : (const void *)csr_pass_kernel<1>;
  cudaError_t e = ensure_smem_attr(fn, smem);
  if (e != cudaSuccess) return e;
  if (mode == 0)
    csr_pass_kernel<0><<<grid, kCsrThreads, smem, s>>>(rp, col, val, m, b, x, part, r2_part, npad,
                                                       gate, bscale, rout);
  else
    csr_pass_kernel<1><<<grid, kCsrThreads, smem, s>>>(rp, col, val, m, b, x, part, r2_part, npad,
                                                       gate, bscale, rout);
  return cudaGetLastError();
}

}  // namespace lsq

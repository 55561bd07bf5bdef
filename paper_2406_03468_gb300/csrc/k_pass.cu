// The two streaming passes over A of the refinement loop (Alg. 1):
//   pass_resid:  r = b - A x,  g = A^T r,  ||r||^2       (refinement RHS)
//   pass_atax:   h = A^T (A z)                           (inner operator)
// Each reads A exactly once.  One warp owns one row at a time: 16-byte
// streaming loads (evict-first; A is far larger than L2), the row dot
// product is reduced with warp shuffles, and the same registers then feed
// the A^T update into per-lane column accumulators.  Rows are split into
// contiguous ranges, one per CTA (2 CTAs per SM); each CTA writes one
// partial n-vector and a separate kernel sums the partials in a fixed order,
// so the result does not depend on scheduling.
#include "lsq_common.cuh"

namespace lsq {

namespace {

template <int NC, bool VEC>
__device__ __forceinline__ void load_row(const double *__restrict__ row, int n, int lane,
                                         double (&a)[2 * NC]) {
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    if (VEC && col + 1 < n) {
      const double2 v = __ldcs(reinterpret_cast<const double2 *>(row + col));
      a[2 * k] = v.x;
      a[2 * k + 1] = v.y;
    } else {
      a[2 * k] = (col < n) ? __ldcs(row + col) : 0.0;
      a[2 * k + 1] = (col + 1 < n) ? __ldcs(row + col + 1) : 0.0;
    }
  }
}

template <int NC>
__device__ __forceinline__ void load_vec(const double *__restrict__ x, int n, int lane,
                                         double (&v)[2 * NC]) {
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    v[2 * k] = (col < n) ? x[col] : 0.0;
    v[2 * k + 1] = (col + 1 < n) ? x[col + 1] : 0.0;
  }
}

// Deterministic CTA reduction of the per-lane column accumulators into part[blockIdx.x].
template <int NC>
__device__ __forceinline__ void cta_store_partial(const double (&h)[2 * NC], double *sh,
                                                  double *__restrict__ part, int npad) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) sh[i] = 0.0;
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        sh[64 * k + 2 * lane] += h[2 * k];
        sh[64 * k + 2 * lane + 1] += h[2 * k + 1];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npad; i += blockDim.x) part[(size_t)blockIdx.x * npad + i] = sh[i];
}

template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    atax_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                const double *__restrict__ z, double *__restrict__ part, int npad,
                const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  __shared__ double sh[NC * 64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  double zr[2 * NC], h[2 * NC];
  load_vec<NC>(z, n, lane, zr);
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) h[k] = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) t = fma(a[k], zr[k], t);
    t = warp_sum(t);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) h[k] = fma(a[k], t, h[k]);
  }
  cta_store_partial<NC>(h, sh, part, npad);
}

template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    resid_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                 const double *__restrict__ b, const double *__restrict__ x,
                 double *__restrict__ part, double *__restrict__ r2_part, int npad) {
  __shared__ double sh[NC * 64];
  __shared__ double r2sh[kPassThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  double xr[2 * NC], g[2 * NC];
  load_vec<NC>(x, n, lane, xr);
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) g[k] = 0.0;
  double r2 = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) s = fma(a[k], xr[k], s);
    s = warp_sum(s);
    const double r = b[i] - s;
    r2 = fma(r, r, r2);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) g[k] = fma(a[k], r, g[k]);
  }
  if (lane == 0) r2sh[warp] = r2;
  cta_store_partial<NC>(g, sh, part, npad);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += r2sh[w];
    r2_part[blockIdx.x] = s;
  }
}

__global__ void reduce_kernel(const double *__restrict__ part, int grid, int npad, int n,
                              const double *__restrict__ scale, double *__restrict__ out,
                              const double *__restrict__ r2_part, double *r2,
                              const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    double s = 0.0;
    for (int g = 0; g < grid; g++) s += part[(size_t)g * npad + j];
    out[j] = scale ? scale[j] * s : s;
  }
  if (r2 != nullptr && j == 0) {
    double s = 0.0;
    for (int g = 0; g < grid; g++) s += r2_part[g];
    *r2 = s;
  }
}

bool vec_ok(const double *A, int64_t lda) {
  return ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 2 == 0);
}

}  // namespace

#define LSQ_PASS_SWITCH(NPAD, ...)             \
  switch ((NPAD) / 64) {                       \
    case 1: { constexpr int NC = 1; __VA_ARGS__; break; }   \
    case 2: { constexpr int NC = 2; __VA_ARGS__; break; }   \
    case 4: { constexpr int NC = 4; __VA_ARGS__; break; }   \
    case 8: { constexpr int NC = 8; __VA_ARGS__; break; }   \
    case 16: { constexpr int NC = 16; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;     \
  }

cudaError_t launch_pass_atax(const double *A, int64_t lda, int64_t m, int n, const double *z,
                             double *part, int grid, int npad, const DevState *gate,
                             cudaStream_t s) {
  const bool vec = vec_ok(A, lda);
  LSQ_PASS_SWITCH(npad, {
    if (vec) atax_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, z, part, npad, gate);
    else atax_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, z, part, npad, gate);
  });
  return cudaGetLastError();
}

cudaError_t launch_pass_resid(const double *A, int64_t lda, int64_t m, int n, const double *b,
                              const double *x, double *part, double *r2_part, int grid, int npad,
                              cudaStream_t s) {
  const bool vec = vec_ok(A, lda);
  LSQ_PASS_SWITCH(npad, {
    if (vec) resid_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, part, r2_part, npad);
    else resid_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, part, r2_part, npad);
  });
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *part, int grid, int npad, int n, const double *scale,
                          double *out, const double *r2_part, double *r2, const DevState *gate,
                          cudaStream_t s) {
  const int th = 128;
  const int blocks = (n + th - 1) / th;
  reduce_kernel<<<blocks, th, 0, s>>>(part, grid, npad, n, scale, out, r2_part, r2, gate);
  return cudaGetLastError();
}

}  // namespace lsq

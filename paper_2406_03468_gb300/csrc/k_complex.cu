// Complex problems (the Prony experiment: A in C^{m x n}, b in C^m) as the
// real least-squares problem of their real embedding.  For a complex row-
// major A with (re, im) interleaved, E (2m x 2n, row-major) has
//   E[2i][2k] = Re a_ik,  E[2i][2k+1] = -Im a_ik,
//   E[2i+1][2k] = Im a_ik, E[2i+1][2k+1] = Re a_ik,
// so that E x_r is A x with real and imaginary parts interleaved: the
// interleaved storage of b and x is already the embedded right-hand side
// and unknown, and min ||b - A x|| over C^n is min ||b_r - E x_r|| over
// R^{2n} (same minimiser).  One streaming pass: 16 bytes read, 32 written
// per complex entry.
#include "lsq_common.cuh"

namespace lsq {

namespace {

__global__ void __launch_bounds__(256)
    embed_complex_kernel(const double2 *__restrict__ A, int64_t lda, int64_t m, int n,
                         double *__restrict__ E) {
  const int64_t lde = 2 * (int64_t)n;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const double2 *row = A + i * lda;
    double *e0 = E + 2 * i * lde, *e1 = e0 + lde;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double2 a = __ldcs(row + k);
      __stcs(reinterpret_cast<double2 *>(e0 + 2 * k), make_double2(a.x, -a.y));
      __stcs(reinterpret_cast<double2 *>(e1 + 2 * k), make_double2(a.y, a.x));
    }
  }
}

}  // namespace

cudaError_t launch_embed_complex(const double *A, int64_t lda, int64_t m, int n, double *E,
                                 int nsm, cudaStream_t s) {
  const int64_t grid = m < (int64_t)nsm * 16 ? m : (int64_t)nsm * 16;
  embed_complex_kernel<<<(unsigned)(grid > 0 ? grid : 1), 256, 0, s>>>(
      reinterpret_cast<const double2 *>(A), lda, m, n, E);
  return cudaGetLastError();
}

}  // namespace lsq

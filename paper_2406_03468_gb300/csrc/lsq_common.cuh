// Internal declarations shared by the CUDA translation units of liblsq.
// Nothing here is part of the C ABI (include/lsq.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsq.h"

namespace lsq {

constexpr double kU = 1.1102230246251565e-16;  // unit roundoff of IEEE double, 2^-53
// u of Alg. 4's step-2 backward-error test: the value Sec. 1.4 states for
// double precision (about 2e-16, 2^-52); at 2^-53 the bound sits at the
// estimate of the correctly rounded solution itself
constexpr double kUKwStop = 2.220446049250313e-16;
constexpr int kPassThreads = 256;               // threads per CTA of the streaming passes
constexpr int kPassCtasPerSm = 2;
constexpr int kCsrCtasPerSm = 5;                // CTAs per SM of a sparse plan's pass grid
constexpr int kVecThreads = 1024;               // threads of the single-CTA vector kernels
constexpr int kMaxZeta = 32;

// Device-resident scalars of one solve.  Kernels of the inner loop read
// `done` first and return at once when it is set, so the host may enqueue a
// few iterations ahead of the stopping decision.
struct DevState {
  double normest, condest;
  double thresh1;        // step-1 stop threshold
  double alpha, beta;    // Polyak coefficients
  double dnorm2;         // ||Delta||^2 of the last inner update
  double rho;            // CG: r^T r
  double r2;             // ||b - A x||^2 of the last residual pass
  double x0norm2;        // ||x0||^2 (scaled coordinates)
  double cnorm2[LSQ_MAX_REFINE];
  int done;              // inner loop of the current step has stopped
  int iters;             // inner updates in the current step
  int max_iters;         // cap of the current step
  int use_thresh;        // 1: stop when ||Delta|| <= thresh1
  int err;               // device-side error (LSQ_ERR_TIMEOUT)
  int nonfinite;         // NaN / Inf seen in A or b
  int zero_col;          // a column norm is zero
  int q2;                // batched solves: the step-2 update count (Theorem 7.1's q0 - 1)
  // LSQR (LSQR-based SPIR): the bidiagonalisation's alpha, beta, the
  // rotation's phibar, rhobar, the next pass's coefficient of s, and the
  // last pass's ||s||^2
  double lq_alpha, lq_beta, lq_phibar, lq_rhobar, lq_bscale, lq_b2;
  // sketched Karlson-Walden estimate (Alg. 4's step-2 test): ||b||^2, and
  // for the iterate checked ||x||^2 (scaled coordinates), ||r||^2, the
  // factor theta / sqrt(1 + theta^2 ||x||^2), ||R_lam^-T g||^2, the estimate
  double bnorm2, kw_xn2, kw_r2, kw_pref, kw_y2, kw_est;
};

// One problem of a batch solved in lockstep (lsq_batch.cu): its sizes, the
// caller's A, b, x and its slices of the batch workspace.  The table of
// items lives in device memory; every batched kernel reads its item from it.
struct BItem {
  const double *A, *b;  // caller's A (m x n, row-major, lda = n) and b (m), device
  double *x;            // caller's x (n), device
  int64_t m;
  int n, npad, d, ld32;
  int method;           // 0: FOSSILS, 1: SPIR
  int cta0, ncta;       // the item's CTAs in the row-parallel launches
  uint64_t seed;
  double eta, alpha, beta;  // distortion and Polyak coefficients (Sec. 2.3, 4.2)
  double *SAb, *W, *part, *r2part, *dcol, *dinv, *Rcm, *Rrm, *rinv, *Dt, *t, *vhead;
  double *xs, *xo, *c, *g, *dy, *dyold, *z, *h, *w, *res, *p;
  float *Ahi, *Alo;     // hi / lo FP32 planes (m x ld32)
  DevState *st;
  int *qflag;           // QR: per-column ready flags (n)
  int qcta0, qncta;     // the item's CTAs in the batched QR launch
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread gets the result.  `scratch` needs
// blockDim.x / 32 doubles of shared memory.  Fixed order for a fixed blockDim.
__device__ __forceinline__ double block_sum(double v, double *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; w++) s += scratch[w];
  return s;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Split for the hi / lo FP32 planes of A (written by the sketch pass or by
// the first residual pass).
// a = hi + lo exactly up to 2^-48 |a|, with integer operations only:
// hi = a rounded to 24 significant bits (round half up, the carry going into
// the exponent as in IEEE), lo = the signed 30-bit remainder scaled by
// 2^(E-52) and rounded to FP32.  Entries outside FP32's normal range give 0
// (the host takes this path only when every column norm is in [2^-40, 2^40]).
__device__ __forceinline__ void split_rn(double a, float &hi, float &lo) {
  const unsigned hw = (unsigned)__double2hiint(a), lw = (unsigned)__double2loint(a);
  const int ef = (int)((hw >> 20) & 0x7ffu) - 896;
  const unsigned sign = hw & 0x80000000u;
  const unsigned up = (lw >> 28) & 1u;
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const unsigned hib = sign | (((unsigned)ef << 23) + m23 + up);
  const int rem = (int)(lw & 0x1fffffffu) - (up ? (1 << 29) : 0);
  const int lf = ef - 52;
  const float l = __fmul_rn(__int2float_rn(rem), __int_as_float((lf > 0 ? lf : 1) << 23));
  hi = (ef > 0 && ef < 254) ? __uint_as_float(hib) : 0.0f;
  lo = (lf > 0 && ef < 254) ? __uint_as_float(__float_as_uint(l) ^ sign) : 0.0f;
}

// cudaFuncSetAttribute(fn, MaxDynamicSharedMemorySize, bytes) once per
// (device, kernel, size): the call costs host time, and the inner loop
// launches its pass dozens of times per solve (lsq_api.cu).
cudaError_t ensure_smem_attr(const void *fn, int bytes);

// Message returned by lsq_last_error() on the calling thread (lsq_api.cu).
void set_last_error(const char *msg);

// Plan internals used by the request server (lsq_server.cu).
// Point a plan at a new problem within the capacity it was created with.
lsq_status plan_configure(lsq_plan P, const lsq_options *opt);
// Run a FOSSILS (method 0) or SPIR (method 1) solve on the plan.
lsq_status plan_solve(lsq_plan P, int method, const double *dA, const double *db, double *dx,
                      lsq_info *info);
// 1: factor the sketch with one launch per column (no cooperative launch).
void plan_set_stepwise_qr(lsq_plan P, int on);

// ---------------------------------------------------------------- launchers
// Every launcher enqueues on `s` and returns the launch's cudaError_t.

// Sparse sign pattern (Philox4x64-10 spec): rows (m x zeta), signbits (m).
cudaError_t launch_sketch_pattern(int64_t m, int d, int zeta, uint64_t seed, int32_t *rows,
                                  uint32_t *signbits, cudaStream_t s);
// Unscaled +-1 sketch of [A b] into SAb (d x (n+1), row-major, must be
// zeroed first) and column sums of squares partials (grid x npad).
// Ahi != NULL: also write the hi / lo FP32 planes of A (m x ld32 floats each,
// ld32 even; hi = A rounded to FP32, lo = the remainder) as the rows stream.
cudaError_t launch_sketch(const double *A, int64_t lda, int64_t m, int n, const double *b,
                          int d, int zeta, const int32_t *rows, const uint32_t *signbits,
                          double *SAb, double *colsq_part, int grid, int npad, float *Ahi,
                          float *Alo, int64_t ld32, cudaStream_t s);
// Gather form of the sketch.  Per plan: source lists of the sketch rows
// (CSR by row h: ptr d + 1 entries, src m zeta entries i | sign << 31 sorted
// by i when no list exceeds sketch_list_max(); cnt: d ints of scratch; *lmax
// = longest list).  Per solve: launch_sketch_prep (column sums of squares,
// largest exponents colexp[0..n) and of b at colexp[npad], FP32 planes),
// then launch_sketch_gather (64-bit fixed-point sums into SAb, d x (n+1)
// row-major, no zeroing needed; cshift / cpow: npad + 1 entries of scratch).
// A may come in row chunks, each taken by a prep then a gather in row order,
// accumulate = 0 for the first: the prep is given the chunk (A, b, Ahi, Alo
// offset to its first row, m its rows), the gather all of A and b and the
// chunk's row range; each chunk gets its own fixed-point scale.  The rows'
// fixed-point values go to Q (>= row1 rows of ldq int64, ldq even; required)
// and Qb (b's, when b is given) first (grid CTAs), once per entry, and the
// gather adds those.
cudaError_t launch_sketch_lists(const int32_t *rows, const uint32_t *signbits, int64_t m, int zeta,
                                int d, int *cnt, int64_t *ptr, uint32_t *src, int *lmax,
                                cudaStream_t s);
int sketch_list_max();
cudaError_t launch_sketch_prep(const double *A, int64_t lda, int64_t m, int n, const double *b,
                               double *colsq_part, int grid, int npad, int *colexp, float *Ahi,
                               float *Alo, int64_t ld32, cudaStream_t s, int accumulate);
cudaError_t launch_sketch_gather(const double *A, int64_t lda, int n, const double *b, int d,
                                 int npad, const int64_t *ptr, const uint32_t *src,
                                 const int *colexp, const int *lmax, int *cshift, double *cpow,
                                 double *SAb, DevState *st, cudaStream_t s, int64_t row0,
                                 int64_t row1, int accumulate, long long *Q, long long *Qb,
                                 int64_t ldq, int grid);
// Column norms from partials, scaling, transpose into column-major W (ld d).
cudaError_t launch_sketch_finalize(const double *colsq_part, int grid, int npad, int n, int d,
                                   int zeta, int col_scale, const double *SAb, double *W,
                                   double *dcol, double *dinv, DevState *st, cudaStream_t s);
// Householder QR of W (d x (n+1), column-major) in place (cooperative).
// ncols = n + number of augmented columns (right-hand sides).
// Cooperative Householder QR of W (d x ncols, column-major), reflectors for
// columns 0..n-1.  vhead: 2 n doubles (u_1, beta per reflector); flags: n ints,
// flag k set to epoch when reflector k is published (epoch != 0, different
// from the previous launch's).  Waits are bounded by timeout_ns.
// Sparse A in CSR form (k_csr.cu): the structure / value check (flags in
// st), the scatter sketch with column sums of squares (partials as the dense
// sketch's), and the passes: mode 0 inner (column sums of a_i (a_i . x)),
// mode 1 residual (v = bs b - A x, rout, ||v||^2 partials, column sums of
// a_i v_i); partials as the dense passes' (grid x npad).
cudaError_t launch_csr_check(const int64_t *rp, const int32_t *col, const double *val, int64_t m,
                             int n, int64_t nnz, const double *b, DevState *st, int nsm,
                             cudaStream_t s);
cudaError_t launch_csr_sketch(const int64_t *rp, const int32_t *col, const double *val, int64_t m,
                              int n, const double *b, int d, int zeta, const int32_t *rows,
                              const uint32_t *signbits, double *SAb, double *colsq_part, int grid,
                              int npad, cudaStream_t s);
cudaError_t launch_csr_pass(int mode, const int64_t *rp, const int32_t *col, const double *val,
                            int64_t m, const double *b, const double *x, double *part,
                            double *r2_part, int grid, int npad, const DevState *gate,
                            const double *bscale, double *rout, cudaStream_t s);
// Real embedding of a complex m x n row-major A (lda complex entries per row,
// (re, im) interleaved, 16-byte aligned) into E (2m x 2n, row-major).
cudaError_t launch_embed_complex(const double *A, int64_t lda, int64_t m, int n, double *E,
                                 int nsm, cudaStream_t s);
// With qb (and n, d in qr_blocked_ok's range) the blocked form of
// k_qr_blocked.cu runs instead: same outputs, panels on qb->sp.
struct QrBlocked {
  double *tws;          // qr_blocked_tws(n) doubles: T of every panel
  cudaStream_t sp;      // the panel stream (high priority)
  cudaEvent_t ev[5];    // ordering events, timing disabled
};
cudaError_t launch_qr(double *W, int d, int n, int ncols, double *vhead, int *flags, int epoch,
                      DevState *st, int grid, uint64_t timeout_ns, cudaStream_t s,
                      const QrBlocked *qb = nullptr);
bool qr_blocked_ok(int d, int n);
size_t qr_blocked_tws(int n);
cudaError_t launch_qr_blocked(double *W, int d, int n, int ncols, double *vhead, double *tws,
                              DevState *st, uint64_t timeout_ns, cudaStream_t s, cudaStream_t sp,
                              cudaEvent_t *ev);
int qr_grid(int ncols, int nsm);       // CTAs of launch_qr
int qr_step_grid(int ncols, int nsm);  // CTAs of launch_qr_stepwise
// The same factorisation as n + 1 ordinary launches (no inter-CTA waits): safe
// to run concurrently with other solves' kernels.
cudaError_t launch_qr_stepwise(double *W, int d, int n, int ncols, double *vhead, int grid,
                               cudaStream_t s);
// R (upper n x n of W) to Rcm / Rrm, 1/R_ii, t = W[0:n, n:n+nb] (column-major n x nb).
cudaError_t launch_extract_r(const double *W, int d, int n, int nb, double *Rcm, double *Rrm,
                             double *rinv, double *t, cudaStream_t s);
// condest / normest of R by power and inverse power iteration.
cudaError_t launch_condest(const double *Rcm, const double *Rrm, const double *rinv,
                           const double *Dt, int n, int iters, DevState *st, cudaStream_t s);
// Dt (2 ceil(n/32) 1024 doubles): the diagonal 32 x 32 blocks of R for both
// solve directions with each entry scaled by 1 / R_ll of the row it updates
// (the triangular solves run the block chains on these).
cudaError_t launch_diag_tiles(const double *Rcm, const double *Rrm, const double *rinv, int n,
                              double *Dt, cudaStream_t s);
// Triangular solve on one CTA.  trans 0: R x = y, 1: R^T x = y.
//   y_eff = y (* in_scale if given); sol = solution;
//   accum != NULL:   accum += sol, out = accum, out_scaled = out_scale * accum
//   accum == NULL:   out = sol, out_scaled = out_scale * sol  (outputs may be NULL)
//   norm2_out != NULL: *norm2_out = ||out||^2
//   gate != NULL: return at once when gate->done.
//   batch > 1: CTA b solves the vectors at offset b * bstride (norm2_out[b]).
//   batch == 1 (n > 96): a cluster of 8 CTAs; a wait that times out sets
//   *err (if given) to LSQ_ERR_TIMEOUT.
cudaError_t launch_trsv(const double *Rcm, const double *Rrm, const double *rinv, const double *Dt,
                        int n, int trans,
                        const double *y, const double *in_scale, double *out,
                        const double *out_scale, double *out_scaled, double *accum,
                        double *norm2_out, const DevState *gate, cudaStream_t s, int batch = 1,
                        int64_t bstride = 0, int *err = nullptr);
// Fused passes (partials: grid x npad doubles, r2_part: grid doubles).
cudaError_t launch_pass_atax(const double *A, int64_t lda, int64_t m, int n, const double *z,
                             double *part, int grid, int npad, const DevState *gate,
                             cudaStream_t s);
// As launch_pass_atax with the row products on the FP32 pipe (k_pass.cu);
// col_exp: A's entries are below 2^col_exp and every column norm is above
// 2^(col_exp - 20).
cudaError_t launch_pass_atax_eft(const double *A, int64_t lda, int64_t m, int n, const double *z,
                                 int col_exp, double *part, int grid, int npad,
                                 const DevState *gate, cudaStream_t s);
// FP32 inner pass of the mixed-precision tier: h = A32^T (A32 z) with FP32
// products and FP32 column sums flushed into FP64 every 32 rows; rows staged
// by TMA bulk copies (ld32 a multiple of 4, A32 16-byte aligned).  err:
// LSQ_ERR_TIMEOUT if a copy never landed.
cudaError_t launch_pass_atax32(const float *A32, int64_t ld32, int64_t m, int n, const double *z,
                               double *part, int grid, int npad, const DevState *gate, int *err,
                               cudaStream_t s);
// Inner pass on the hi / lo FP32 planes: row and column sums both in
// double-float on the FP32 pipe (column sums flushed into FP64 every 8 rows);
// rows staged by TMA bulk copies.  ld32: a multiple of 4 (16-byte rows);
// Ahi / Alo 16-byte aligned.  err: LSQ_ERR_TIMEOUT if a copy never landed.
// batch > 1: grid rows c < batch work on z + c zstride into part + c pstride.
cudaError_t launch_pass_atax_df(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                                const double *z, double *part, int grid, int npad,
                                const DevState *gate, int *err, cudaStream_t s, int batch = 1,
                                int64_t zstride = 0, int64_t pstride = 0);
// Many right-hand sides in one read of the hi / lo planes (k_multi_df.cu):
// the partial sums of H = A^T (A Z) for k <= 64 vectors (Z n x k column-
// major), CTA g's for vector c at part + (c grid + g) npad.  Needs n <= 256,
// ld32 % 4 == 0 and one CTA per SM of shared memory (multi_df_supported).
bool multi_df_supported(int n, int k, int64_t ld32);
cudaError_t launch_pass_atax_df_multi(const float *Ahi, const float *Alo, int64_t ld32, int64_t m,
                                      int n, const double *Z, int k, double *part, int grid,
                                      int npad, const DevState *gate, int *err, cudaStream_t s);
// out (n x batch, column-major) = scale .* the sums of a batched pass's partials.
cudaError_t launch_reduce_batched(const double *part, int grid, int npad, int n, int batch,
                                  const double *scale, double *out, const DevState *gate,
                                  cudaStream_t s);
// Residual pass r = b - A x, partials of A^T r and of ||r||^2, all FP64.
// (A^T r is a sum with heavy cancellation -- r is nearly orthogonal to
// range(A) -- and its rounding reaches x through kappa^2, so it stays FP64.)
// Ahi != NULL: also write the hi / lo FP32 planes of A (as launch_sketch).
// bscale != NULL: r = (*bscale) b - A x; rout != NULL: r is written there
// (rout may equal b); gate: return at once when gate->done (LSQR's pass).
cudaError_t launch_pass_resid(const double *A, int64_t lda, int64_t m, int n, const double *b,
                              const double *x, double *part, double *r2_part, int grid, int npad,
                              cudaStream_t s, float *Ahi = nullptr, float *Alo = nullptr,
                              int64_t ld32 = 0, const DevState *gate = nullptr,
                              const double *bscale = nullptr, double *rout = nullptr);
// Compensated residual pass (Dot2): r = b - A' x and the (sum, error) pairs of
// A'^T r per CTA into part2 (grid x 2 npad), ||r||^2 partials, with
// A' = fl(A diag(cs)) when cs is non-NULL, else A; reduce_dot2 adds the pairs
// with TwoSum (scale may be NULL).
cudaError_t launch_pass_resid_dot2(const double *A, int64_t lda, int64_t m, int n,
                                   const double *b, const double *x, const double *cs,
                                   double *part2, double *r2_part, int grid, int npad,
                                   cudaStream_t s);
cudaError_t launch_reduce_dot2(const double *part2, int grid, int npad, int n, const double *scale,
                               double *out, const double *r2_part, double *r2, cudaStream_t s);
// out[j] = scale[j] * sum_g part[g][j] (scale may be NULL); r2 (if non-NULL)
// = sum_g r2_part[g]; gated.
cudaError_t launch_reduce(const double *part, int grid, int npad, int n, const double *scale,
                          double *out, const double *r2_part, double *r2, const DevState *gate,
                          cudaStream_t s);
int pass_npad(int n);

// Many right-hand sides (k_multi.cu): DMMA row-block passes and per-column steps.
int multi_np8(int n);
bool multi_supported(int n, int k);
cudaError_t launch_multi_atax(const double *A, int64_t lda, int64_t m, int n, int k,
                              const double *Z, double *part, int grid, const DevState *gate,
                              cudaStream_t s);
cudaError_t launch_multi_resid(const double *A, int64_t lda, int64_t m, int n, int k,
                               const double *B, int64_t ldb, const double *X, double *part,
                               double *r2part, int grid, cudaStream_t s);
cudaError_t launch_multi_reduce(const double *part, int grid, int n, int k, const double *scale,
                                double *out, const double *r2part, double *r2,
                                const DevState *gate, cudaStream_t s);
cudaError_t launch_multi_polyak(int n, int k, const double *C, const double *Wv, double *DY,
                                double *DYold, double *dn2, const double *thresh, DevState *st,
                                cudaStream_t s);
cudaError_t launch_multi_init(int n, int k, const double *C, double *DY, double *DYold,
                              int max_iters, int use_thresh, DevState *st, cudaStream_t s);
cudaError_t launch_multi_thresh(int k, double gamma, double rho, const double *x0n2,
                                const double *r2, double *thresh, const DevState *st,
                                cudaStream_t s);
cudaError_t launch_sketch_b_to_w(const double *SBb, int d, int n, int k, int zeta, double *W,
                                 DevState *st, cudaStream_t s);
cudaError_t launch_cm_to_rm(const double *Xcm, int n, int k, double *X, cudaStream_t s);

// LSQR-based SPIR (k_lsqr.cu).  One pass: s <- (*bscale) s - A z, partials
// of A^T s and ||s||^2, on the hi / lo planes in double-float (the FP64 form
// is launch_pass_resid with bscale and rout = s); gated.
cudaError_t launch_pass_lsqr_df(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                                const double *z, double *s, const double *bscale, double *part,
                                double *r2part, int grid, int npad, const DevState *gate, int *err,
                                cudaStream_t st);
// LSQR start from c = R^{-T} D^{-1} A^T r_i (||c||^2 = st->cnorm2[step],
// ||r_i||^2 = st->r2): v = w = c / ||c||, dy = 0, the scalars in st.
cudaError_t launch_lsqr_init(int n, const double *c, int step, double *v, double *w, double *dy,
                             int max_iters, int use_thresh, DevState *st, cudaStream_t s);
// One LSQR iteration from p = R^{-T} D^{-1} A^T s and st->lq_b2 (gated).
cudaError_t launch_lsqr_update(int n, const double *p, double *v, double *w, double *dy,
                               DevState *st, cudaStream_t s);

// Batched phases (lsq_batch.cu): every launch covers all `count` items of
// the table; row-parallel launches take `grid` CTAs, CTA g working on item
// cta_item[g].  Kernels of the inner loop return at once for an item whose
// st->done is set.
// Kernel attributes of the batched kernels for n <= nmax (before any capture).
cudaError_t prepare_b_kernels(int nmax);
cudaError_t prepare_b_inner();
cudaError_t launch_b_zero(const BItem *items, int count, cudaStream_t s);  // SAb = 0
// Re-deal the row-parallel CTAs over all items (all = 1) or over the items
// whose inner loop runs (all = 0); each item's partials hold grid entries.
cudaError_t launch_b_redeal(BItem *items, int count, int *cta_item, int grid, int all,
                            cudaStream_t s);
cudaError_t launch_b_sketch(const BItem *items, const int *cta_item, int grid, int zeta,
                            cudaStream_t s);
cudaError_t launch_b_finalize(const BItem *items, int count, int zeta, cudaStream_t s);
// QR of every item's sketch in one cooperative launch (the flag form of
// launch_qr, item i on CTAs qcta0 .. qcta0 + qncta - 1 of the grid, qmap the
// CTA -> item map, -1 for none); at most b_qr_max_ctas CTAs, at least
// b_qr_min_ctas(n) per item.
cudaError_t launch_b_qr(const BItem *items, const int *qmap, int grid, int epoch,
                        uint64_t timeout_ns, cudaStream_t s);
int b_qr_max_ctas(int nsm);
int b_qr_min_ctas(int n);
// QR of every item's sketch, one launch per column step k = -1 .. nmax - 1
// (qcta CTAs per item).
cudaError_t launch_b_qr_step(const BItem *items, int count, int qcta, int k, cudaStream_t s);
// R, 1/R_ii, t, the scaled diagonal tiles, condest / normest, x0 and the
// step-2 count q2 (into st->max_iters of the item's state, read by b_init).
cudaError_t launch_b_setup(const BItem *items, int count, int cond_iters, int max_inner,
                           int nmax, cudaStream_t s);
// mode 0: z = D^-1 R^-1 (dy or p) (gated); 1: w = R^-T h (gated);
// 2: c = R^-T g and ||c||^2 into st->cnorm2[step]; 3: xs += R^-1 dy, xo = D^-1 xs.
cudaError_t launch_b_trsv(const BItem *items, int count, int mode, int step, int nmax,
                          cudaStream_t s);
cudaError_t launch_b_resid(const BItem *items, const int *cta_item, int grid, cudaStream_t s);
cudaError_t launch_b_inner(const BItem *items, const int *cta_item, int grid, cudaStream_t s);
// mode 0: g = D^-1 sum of the residual partials, st->r2; 1: h (gated).
cudaError_t launch_b_reduce(const BItem *items, int count, int nmax, int mode, cudaStream_t s);
// Step thresholds (step 0) and the inner solver's start for step `step`.
cudaError_t launch_b_init(const BItem *items, int count, int step, int max_inner, double gamma,
                          double rho, cudaStream_t s);
cudaError_t launch_b_update(const BItem *items, int count, cudaStream_t s);
cudaError_t launch_b_copy_x(const BItem *items, int count, cudaStream_t s);

// Sketched Karlson-Walden estimate (k_vec.cu).  launch_bnorm2: st->bnorm2 =
// ||b||^2.  launch_kw_build: W2 (2n x n, column-major) = [R; sqrt(lam) I]
// with lam = theta^2 ||r||^2 / (1 + theta^2 ||x||^2), theta^2 = ||A D^-1||_F^2
// / ||b||^2 (st->kw_r2; ||x||^2 of xs, the scaled x, into st->kw_xn2), and
// st->kw_pref.  launch_kw_finish:
// st->kw_est = kw_pref sqrt(kw_y2).  launch_scale_vec: y = s .* x.
cudaError_t launch_bnorm2(const double *b, int64_t m, DevState *st, cudaStream_t s);
cudaError_t launch_kw_build(const double *Rcm, int n, const double *dcol, const double *dinv,
                            const double *xs, double *W2, DevState *st, cudaStream_t s);
cudaError_t launch_kw_finish(DevState *st, cudaStream_t s);
cudaError_t launch_scale_vec(int n, const double *sc, const double *x, double *y, cudaStream_t s);

// Inner-solver kernels (single CTA).
cudaError_t launch_inner_init(int method, int n, const double *c, double *dy, double *dy_old,
                              double *res, double *p, int max_iters, int use_thresh,
                              DevState *st, cudaStream_t s);
cudaError_t launch_polyak_update(int n, const double *c, const double *w, double *dy,
                                 double *dy_old, DevState *st, cudaStream_t s);
cudaError_t launch_cg_update(int n, const double *q, double *p, double *res, double *dy,
                             DevState *st, cudaStream_t s);
// thresh1 = u (gamma normest ||x0|| + rho condest sqrt(r2)); records cnorm2[0].
cudaError_t launch_set_thresh(double gamma, double rho, DevState *st, cudaStream_t s);

}  // namespace lsq

/*
 * lsq.h -- C ABI of the GB300 (sm_103a) least-squares library: FOSSILS and
 * SPIR, the backward-stable randomized solvers of Epperly, Meier and
 * Nakatsukasa (arXiv 2406.03468), for min ||b - A x||_2 with A tall and
 * dense (m >> n).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Layout     A is m x n, row-major, FP64, leading dimension lda >= n (in
 *            doubles).  Vectors are contiguous FP64.  Pointers named d*
 *            are DEVICE pointers on the plan's device; h* are host pointers.
 * Ownership  The caller owns every buffer it passes.  Buffers are borrowed
 *            for the duration of the call only; every entry point returns
 *            after its work on the plan's stream has finished (the solve
 *            entry points wait for the stream).  The plan owns its
 *            workspace (sketch, R, iterates, partial sums), allocated once
 *            at lsq_plan_create and freed by lsq_plan_destroy.
 * Errors     Status codes only; nothing is thrown across the ABI.  After a
 *            status < 0, lsq_last_error() returns a message for the calling
 *            thread.  Device-side waits are bounded: a wait that runs out
 *            returns LSQ_ERR_TIMEOUT instead of hanging.
 * Threads    A plan is used by one thread at a time.  Different plans may be
 *            used concurrently from different threads.
 * CUDA       A CUDA library failure returns LSQ_ERR_CUDA.  There is no CPU
 *            fallback: without a usable GPU every compute call fails.
 */
#ifndef LSQ_H
#define LSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LSQ_OK = 0,
  LSQ_PENDING = 1,               /* lsq_poll: the request is not finished yet */
  LSQ_WARN_RANK_DEFICIENT = 2,   /* solved, but condest > 1/(30u) (Sec. 4.2) */
  LSQ_ERR_INVALID = -1,          /* bad argument (sizes, null pointers, options) */
  LSQ_ERR_OOM = -2,              /* device allocation or admission failed */
  LSQ_ERR_CUDA = -3,             /* a CUDA call failed */
  LSQ_ERR_NOT_CONVERGED = -4,    /* refinement monitor never met its target */
  LSQ_ERR_TIMEOUT = -5,          /* a bounded device-side wait ran out */
  LSQ_ERR_NONFINITE = -6         /* A or b holds NaN or Inf */
} lsq_status;

/* Arithmetic of the inner iterations.  On every path the residual b - A x,
 * A^T r, the update of x, the QR of the sketch and the triangular solves with
 * R are FP64.  The inner passes h = A^T (A z) of the FP64 path run, by
 * default, in double-float on the FP32 pipe over an exact-to-2^-48 split of A
 * into FP32 hi / lo planes (an FP64-class evaluation, within the per-element
 * error bound of an FP64 pass); inner_fp64_fma = 1 makes them strict FP64
 * (two FP64 FMAs per element of A). */
enum {
  LSQ_PREC_AUTO = 0,        /* FP32 inner passes when condest < fp32_cond_max, else the FP64 path */
  LSQ_PREC_FP64 = 1,        /* the FP64 path (inner passes as inner_fp64_fma selects) */
  LSQ_PREC_FP32_INNER = 2   /* inner passes read the FP32 hi plane of A (FP32 arithmetic) */
};

typedef struct lsq_plan_s *lsq_plan;

typedef struct {
  int64_t m, n;          /* problem size, m >= n >= 1, n <= LSQ_MAX_N */
  int64_t lda;           /* leading dimension of A in doubles (0 => n) */
  int32_t d;             /* sketch rows (0 => 12 n), n <= d */
  int32_t zeta;          /* nonzeros per sketch column (0 => 8), 1..32, <= d */
  uint64_t seed;         /* Philox key of the sparse sign embedding */
  double eta;            /* distortion for alpha, beta (0 => sqrt(n/d)) */
  int32_t col_scale;     /* 1: scale columns of A to unit norm (Alg. 4), 0: off */
  int32_t max_inner;     /* cap on inner updates per refinement step (0 => 100) */
  int32_t max_refine;    /* refinement steps (0 => 2 on FP64; FP32 tier: up to 6) */
  int32_t precision;     /* LSQ_PREC_* (default LSQ_PREC_FP64).  With AUTO and
                            FP32_INNER the FP32 tier runs its inner passes on the hi
                            plane of A (A rounded to FP32), the residual, A^T r, x update, QR and
                            triangular solves staying FP64, and refines until ||c_i||
                            stops halving (at least 2, at most max(max_refine, 6) steps) */
  double fp32_cond_max;  /* FP32-inner gate on condest (0 => 1e5) */
  double stop_gamma;     /* step-1 stop constant gamma (Alg. 4: 10; Sec. 4.2 text: 1) */
  double stop_rho;       /* step-1 stop constant rho (Alg. 4: 0.4; Sec. 4.2 text: 0.04) */
  int32_t fixed_inner;   /* > 0: every refinement step runs exactly this many updates */
  int32_t timing;        /* 1: time every streaming pass with CUDA events (lsq_info) */
  int32_t inner_fp64_fma;/* 1: inner pass with two FP64 FMAs per element on A itself.
                            0 (default): the sketch pass also writes exact hi / lo FP32
                            planes of A (8 m n bytes of device memory) and the inner
                            passes run in double-float on the FP32 pipe when every
                            column norm is in [2^-40, 2^40] */
  int32_t nrhs;          /* > 0: plan for lsq_solve_fossils_multi with this many
                            right-hand sides (multiple of 8, <= 64; n <= 256) */
  int32_t qr_wait_us;    /* > 0: each inter-CTA wait of the QR of the sketch gives up
                            after this many microseconds (0 => 5 s); the solve then
                            returns LSQ_ERR_TIMEOUT and the plan stays usable.  The
                            other device waits (TMA copies, cluster transfers) keep
                            their own limits, so no copy can outlive its CTA */
  int32_t kw_stop;       /* 1: end the second refinement step with Alg. 4's test: after
                            inner updates 1, 6, 11, ... the sketched Karlson-Walden
                            estimate of the iterate's backward error (eq. (sketched-kw),
                            theta = ||A D^-1||_F / ||b||) is compared with
                            u ||A D^-1||_F, u = 2^-52 (Sec. 1.4's value for double;
                            2^-53 is the rounding level of the solution itself), and
                            the step stops below it (at most
                            max_inner updates); 0 (default): Theorem 7.1's q0 - 1
                            updates.  Each test costs one compensated FP64 pass over A
                            (about ten times a plain one) and a QR of a 2n x n matrix.
                            The second step's inner passes are then strict FP64
                            (inner_kernel 0): the double-float pass holds A to 2^-48,
                            which leaves that step's answer a few u ||A||_F from
                            backward stable on kappa ~ 1e12 problems, above the bound */
  int32_t sparse;        /* 1: the plan solves CSR matrices (lsq_solve_csr) and allocates
                            no FP32 planes or fixed-point copy of A; precision must be
                            FP64, nrhs and kw_stop 0.  0 (default): dense A */
  int32_t reserved[3];
} lsq_options;

#define LSQ_MAX_N 1024
#define LSQ_MAX_REFINE 8

typedef struct {
  int32_t iters[LSQ_MAX_REFINE];  /* inner updates run in each refinement step */
  int32_t refine_steps;           /* refinement steps run */
  int32_t path;                   /* LSQ_PREC_FP64 or LSQ_PREC_FP32_INNER */
  int32_t passes;                 /* streaming passes over A (sketch + residuals + inner) */
  int32_t status;                 /* same value as the return code */
  double condest;                 /* sigma_max(R) / sigma_min(R) estimate */
  double normest;                 /* sigma_max(R) estimate */
  double cnorm[LSQ_MAX_REFINE];   /* ||c_i|| = ||R^{-T} A^T (b - A x_i)|| per step */
  double resid0;                  /* ||b - A x_0|| (sketch-and-solve) */
  double thresh1;                 /* step-1 stop threshold */
  float ms_sketch, ms_qr, ms_refine, ms_total;  /* device time of the phases */
  int32_t launches;               /* kernels launched by the call (gated no-ops included) */
  int32_t n_inner_pass;           /* timing: inner A^T(A z) passes that did work */
  float ms_inner_pass;            /* timing: their summed device time */
  int32_t n_resid_pass;           /* timing: residual passes */
  float ms_resid_pass;            /* timing: their summed device time */
  float ms_sketch_pass;           /* timing: the sketch pass */
  int32_t inner_kernel;           /* 0: FP64-FMA inner pass, 1: FP32-pipe row products on A,
                                     2: FP32 tier pass (hi plane), 3: double-float pass on
                                     the hi / lo planes (one batched launch for many
                                     right-hand sides), 4: FP64 tensor-core (DMMA)
                                     many-right-hand-side pass, 5: the double-float
                                     pass for many right-hand sides that applies each
                                     row block of A to all k vectors (A read once) */
  double bytes_a;                 /* bytes of A (and its FP32 copy) streamed by the solve */
  double be_sketch_est;           /* kw_stop: the last sketched Karlson-Walden estimate
                                     (absolute; divide by ||A D^-1||_F), else 0 */
} lsq_info;

/* Fill *o with the defaults listed above (m, n, lda left 0). */
void lsq_options_default(lsq_options *o);

/* Create a plan for problems of size opt->m x opt->n on the current CUDA
 * device, working on the given CUDA stream (cudaStream_t; NULL = legacy
 * default stream).  Allocates the whole workspace (device memory) once.
 * Errors: LSQ_ERR_INVALID on bad options, LSQ_ERR_OOM, LSQ_ERR_CUDA. */
lsq_status lsq_plan_create(const lsq_options *opt, void *cuda_stream, lsq_plan *out);

/* Point an existing plan at another problem without allocating: opt->m,
 * opt->n, the sketch size d and zeta must not exceed the plan's (the sizes
 * it was created with), nrhs must match, and AUTO / FP32_INNER precision
 * needs a plan created with one of them.  Errors: LSQ_ERR_INVALID. */
lsq_status lsq_plan_configure(lsq_plan plan, const lsq_options *opt);

/* Free the plan and its workspace.  NULL is ignored. */
void lsq_plan_destroy(lsq_plan plan);

/* Sketch, column scaling and preconditioner (Alg. 1, the lines before the
 * refinement loop; Alg. 4's column scaling): colnorms d_j of A,
 * [SA Sb] = S [A diag(d)^{-1}, b] with S the Philox sparse sign embedding
 * (Sec. 4.2), Householder QR [SA Sb] -> R and t = (Q^T Sb)[0:n],
 * the condest / normest estimates of R, and the sketch-and-solve x0 =
 * R^{-1} t (Sec. 2.3).  Keeps R, t, x0 in the plan.
 * dA: m x n row-major (lda), db: m.  Errors: LSQ_ERR_NONFINITE if A or b is
 * not finite, LSQ_ERR_INVALID for a zero column (with col_scale). */
lsq_status lsq_sketch(lsq_plan plan, const double *dA, const double *db);

/* FOSSILS (Alg. 2 with the stopping rules of Sec. 4.2): lsq_sketch, then
 * refinement steps x_{i+1} = x_i + R^{-1} dy_i with the Polyak heavy ball
 * (Alg. 5) on R^{-T} A^T A R^{-1} dy = c_i.  Writes the solution (original
 * column scaling) to dx (n, device).  info may be NULL.
 * Returns LSQ_OK or LSQ_WARN_RANK_DEFICIENT on success. */
lsq_status lsq_solve_fossils(lsq_plan plan, const double *dA, const double *db, double *dx,
                             lsq_info *info);

/* SPIR (Alg. 3): as lsq_solve_fossils with conjugate gradient (from dy = 0)
 * as the inner solver. */
lsq_status lsq_solve_spir(lsq_plan plan, const double *dA, const double *db, double *dx,
                          lsq_info *info);

/* LSQR-based SPIR (Sec. 4.2, "SPIR: conjugate gradient or LSQR?"): as
 * lsq_solve_spir, with each refinement step's least-squares problem
 * min || r_i - A D^{-1} R^{-1} dy || solved by LSQR (Paige and Saunders)
 * from dy = 0 in place of CG on its normal equations, and SPIR's two
 * stopping rules applied to the LSQR step (phi_k / rho_k) w_k.  One pass
 * over A per LSQR iteration gives both B v and B^T u (the m-vector of the
 * bidiagonalisation, 8 m bytes, is plan workspace).  The inner passes run
 * in double-float on the hi / lo FP32 planes of A (inner_fp64_fma = 1: two
 * FP64 FMAs per element); the FP32 tier is not used (precision AUTO and
 * FP32_INNER take the FP64 path). */
lsq_status lsq_solve_spir_lsqr(lsq_plan plan, const double *dA, const double *db, double *dx,
                               lsq_info *info);

/* FOSSILS (method 0), SPIR (1) or LSQR-based SPIR (2) for a sparse A in CSR
 * form (the paper's SuiteSparse runs, Sec. 5 "Runtime and iteration count",
 * where SPIR uses d = 3n: set opt.d).  The plan must have been created with
 * opt.sparse = 1 for this m, n.  row_ptr: m + 1 int64 with row_ptr[0] = 0 and
 * row_ptr[m] = nnz; col: nnz int32 column indices in [0, n), distinct within
 * a row (any order); val: nnz FP64 values; db: m; dx: n (out); all device
 * pointers, read-only except dx.  The sketch scatters the nonzeros (FP64
 * atomics, so its rounding order is not fixed); the residual and inner
 * passes run in FP64 over the nonzeros, one warp per row, deterministic for
 * a fixed plan.  Everything after the sketch is the dense solve's.
 * Errors: LSQ_ERR_INVALID (NULL, nnz < 0, a structure that is not CSR of an
 * m x n matrix with nnz entries, a zero column, a dense plan),
 * LSQ_ERR_NONFINITE, and those of the dense solve. */
lsq_status lsq_solve_csr(lsq_plan plan, int method, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const double *val, const double *db, double *dx,
                         lsq_info *info);

/* A complex least-squares problem min ||b - A x||, A in C^{m x n}, b in C^m
 * (the paper's Prony experiment, Sec. 5 "Runtime and iteration count", and
 * the first solve of Prony's method in its appendix), by FOSSILS (method 0),
 * SPIR (1) or LSQR-based SPIR (2) applied to the real embedding
 *   E[2i][2k] = Re a_ik, E[2i][2k+1] = -Im a_ik,
 *   E[2i+1][2k] = Im a_ik, E[2i+1][2k+1] = Re a_ik   (E: 2m x 2n),
 * whose least-squares solution is x with real and imaginary parts
 * interleaved, so b and x are passed in their complex storage.
 * plan: created for m_r = 2m, n_r = 2n (n <= LSQ_MAX_N / 2), lda = 0; its
 * options apply to the embedded problem (d = 12 n_r by default; with kw_stop
 * the bound is u ||E D^-1||_F = sqrt(2) u ||A D^-1||_F).
 * dA: m x n complex, row-major, (re, im) interleaved doubles, lda complex
 * entries per row (0 => n), 16-byte aligned; db: m complex; dx: n complex
 * (out); dwork: 2m x 2n doubles (16-byte aligned), caller-owned, overwritten
 * with E.  All device pointers.  info as for the real solves.
 * Errors: LSQ_ERR_INVALID (NULL, odd plan sizes, lda, alignment, method), and
 * those of the real solve. */
lsq_status lsq_solve_complex(lsq_plan plan, int method, const double *dA, int64_t lda,
                             const double *db, double *dx, double *dwork, lsq_info *info);

/* FOSSILS for k = opt.nrhs right-hand sides sharing one sketch S [A B] and
 * one QR (Alg. 1 with the augmented columns Q^T S B; Alg. 2 / Alg. 5 per
 * column, each column with its own Polyak vectors and step-1 threshold, the
 * step ending when every column meets its own).  The residual pass
 * G = A^T (B - A X) is an FP64 tensor-core (DMMA) contraction over row
 * blocks of A.  The inner pass H = A^T (A Z) runs in double-float on the
 * hi / lo planes, each row block of A applied to all k vectors in one read
 * of A.  With inner_fp64_fma = 1, or column norms outside [2^-40, 2^40], it
 * is also a DMMA contraction.  dB: m x k row-major with leading
 * dimension ldb >= k (0 => k); dX: n x k row-major (device).  Requires
 * n <= 256.  info (may be NULL) reports the largest ||c_i|| over columns. */
lsq_status lsq_solve_fossils_multi(lsq_plan plan, const double *dA, const double *dB,
                                   int64_t ldb, double *dX, lsq_info *info);

/* As lsq_solve_fossils / lsq_solve_spir with HOST buffers hA (m x n, lda;
 * (m - 1) lda + n doubles are read), hb (m) and hx (n): copies A and b to
 * plan-owned device memory (allocated on first use, grown when a
 * reconfigured plan needs more, kept with the plan), solves, and copies x
 * back.  method: 0 = FOSSILS, 1 = SPIR, 2 = LSQR-based SPIR.  When the sketch takes its gather
 * form (m n >= 2^24), A is copied in row chunks of at least 128 MB (16 at
 * most) on a copy stream and the sketch of each chunk (Sec. 4.2) runs as it
 * lands, so the sketch overlaps the copy; each chunk's sums get their own
 * fixed-point scale and are added in FP64 in row order, so the sketch, and
 * x, can differ from the device entry's by rounding.  The overlap needs
 * page-locked host memory (else each chunk's copy completes before the call
 * goes on).  Returns after x is in hx. */
lsq_status lsq_solve_host(lsq_plan plan, int method, const double *hA, const double *hb,
                          double *hx, lsq_info *info);

/* ---- step-level entry points (each one step of the path, for composing
 * ---- the path and for checking each step on its own) -------------------- */

/* Rows and signs of S: d_rows (m x zeta int32, device), d_signbits (m
 * uint32, device; bit k set => the k-th nonzero of column j is -1).  The
 * pattern of Sec. 4.2's sparse sign embedding, drawn with Philox4x64-10
 * (Salmon et al. 2011): for column j, key (seed, 0) and counters (j, t, 0,
 * 0), t = 0, 1, ...; each block gives eight 32-bit words, low half first; the
 * first word of block 0 is the sign word, every later word u is a candidate
 * row floor(u d / 2^32), taken unless already drawn, until zeta rows. */
lsq_status lsq_sketch_pattern(lsq_plan plan, int32_t *d_rows, uint32_t *d_signbits);

/* After lsq_sketch: copy the scaled sketch [SA Sb] (d x (n+1), column-major,
 * leading dimension d) and the column norms d_j (n) to device buffers. */
lsq_status lsq_get_sketch(lsq_plan plan, double *dSAb, double *dcolnorm);

/* After lsq_sketch or a solve on the plan: copy the sums of the unscaled
 * sketch, S' [A b] with S' the +-1 pattern of Sec. 4.2's embedding (no
 * zeta^{-1/2}, no column scaling), to dSAb (d x (n+1) FP64, row-major,
 * device).  For m n >= 2^24 these are the 64-bit fixed-point sums, each
 * rounded once to FP64 (for lsq_solve_host: per row chunk, the chunks added
 * in order); below that, FP64 atomic sums whose order is not fixed.
 * Errors: LSQ_ERR_INVALID for NULL arguments or before any sketch. */
lsq_status lsq_get_sketch_raw(lsq_plan plan, double *dSAb);

/* After lsq_sketch: copy R (n x n, row-major, zeros below the diagonal),
 * t = (Q^T Sb)[0:n] and x0 (scaled coordinates) to device buffers (any may
 * be NULL), and the condest / normest estimates to host doubles (may be NULL). */
lsq_status lsq_get_R(lsq_plan plan, double *dR, double *dt, double *dx0, double *condest,
                     double *normest);

/* One fused streaming pass over A: dh = A^T (A dz) (the operator of
 * Sec. 2.1's preconditioned normal equations before the R solves; Alg. 1's
 * Apply), with the inner-pass kernel the solve would use: after lsq_sketch
 * and unless inner_fp64_fma is set, the FP32-pipe row products when the
 * column norms allow it; otherwise two FP64 FMAs per element.  dz, dh: n,
 * device.  No scaling is applied. */
lsq_status lsq_apply_normal(lsq_plan plan, const double *dA, const double *dz, double *dh);

/* Many right-hand sides, one pass: dH = A^T (A dZ) for the plan's k = nrhs
 * vectors (Alg. 1's Apply for each right-hand side of
 * lsq_solve_fossils_multi), with the inner-pass kernel that solve uses.
 * After lsq_solve_fossils_multi on the same A (it writes the hi / lo FP32
 * planes) and unless inner_fp64_fma is set: double-float on the planes,
 * every row block of A applied to all k vectors while it is in shared
 * memory; otherwise the FP64 tensor-core (DMMA) contraction on dA.  dZ, dH:
 * n x k column-major (vector c at offset c n), device.  No scaling is
 * applied.  Errors: LSQ_ERR_INVALID (NULL argument, nrhs = 0 plan). */
lsq_status lsq_apply_normal_multi(lsq_plan plan, const double *dA, const double *dZ, double *dH);

/* The sketched Karlson-Walden estimate (Sec. 4.1, eq. (sketched-kw)) of the
 * backward error of x (dx: n, device, original column scaling) on the
 * column-scaled problem of the plan's last sketch, with theta =
 * ||A D^-1||_F / ||b|| (Sec. 4.2): theta / sqrt(1 + theta^2 ||x_s||^2) *
 * || ((SA)^T SA + lam I)^{-1/2} (A D^-1)^T (b - A x) ||, lam = theta^2
 * ||b - A x||^2 / (1 + theta^2 ||x_s||^2), x_s = D x.  Alg. 4 evaluates it
 * through the SVD of SA; here (SA)^T SA = R^T R and the norm is
 * ||R_lam^{-T} g|| with R_lam the R factor of [R; sqrt(lam) I] (Householder
 * QR of that 2n x n matrix): the same quantity.  The residual b - A x and
 * A^T r are FP64 with compensated (Dot2) sums, so their rounding stays far
 * below the u ||A D^-1||_F level the estimate is compared with.
 * *est: host double, absolute (divide by ||A D^-1||_F, sqrt(n) with column
 * scaling, for the relative value).  Needs lsq_sketch (or a solve) on dA.
 * Errors: LSQ_ERR_INVALID (NULL argument, no sketch). */
lsq_status lsq_sketched_kw(lsq_plan plan, const double *dA, const double *db, const double *dx,
                           double *est);

/* One fused streaming pass over A: dg = A^T (db - A dx) and *r2 = ||b - A x||^2
 * (Alg. 1, the refinement right-hand side before the R^{-T} solve).  r2 is a
 * host pointer and may be NULL. */
lsq_status lsq_residual(lsq_plan plan, const double *dA, const double *db, const double *dx,
                        double *dg, double *r2);

/* Triangular solve with the plan's R by back substitution (Sec. 6): dx =
 * R^{-1} dy (trans = 0) or R^{-T} dy (trans = 1).  dx may equal dy. */
lsq_status lsq_trsv(lsq_plan plan, int trans, const double *dy, double *dx);

/* One fused pass dh = A^T (A dz) that allocates no device memory, for
 * callers that cannot call cudaMalloc: code inside a framework that owns all
 * device memory through its own pool, or a latency-critical loop that cannot
 * afford cudaMalloc's implicit synchronisation or its failure.  The paper
 * has no counterpart; it is a packaging of lsq_apply_normal's FP64 pass.
 * No plan is needed.  dA: m x n row-major (lda, 0 => n), dz, dh: n, all
 * device pointers owned by the caller; cuda_stream: cudaStream_t (NULL =
 * default stream).  Every call synchronizes that stream before it returns.
 * Scratch: a fixed 2 MiB device array inside the library (held by every GPU
 * that loads it until the process exits).  The first call on a device looks
 * up the array's device address and must come before any stream capture.
 * Calls that overlap on the GPU share the array and race.
 * Errors: LSQ_ERR_INVALID for NULL pointers, lda < n or n > LSQ_MAX_N;
 * LSQ_ERR_CUDA when a launch fails. */
lsq_status lsq_apply_normal_noalloc(const double *dA, int64_t m, int64_t n, int64_t lda,
                                    const double *dz, double *dh, void *cuda_stream);

/* ---- batched solves: many small problems in lockstep -------------------- */

/* Many independent problems (n <= 256 each) solved together, every phase of
 * the method one launch over all of them: the sketch, each column step of
 * the QR, the setup after it, and each refinement phase (the launches of
 * each phase captured once in a CUDA graph and replayed).  The paper solves
 * one problem at a time; batching is this library's own, for streams of
 * small problems whose kernels would otherwise last about as long as their
 * launches.  Per item the method is lsq_solve_fossils / lsq_solve_spir's
 * with default options (d = 12 n, zeta = 8, column scaling, two refinement
 * steps, Alg. 4's step-1 stop and Theorem 7.1's step-2 count), except that
 * the sketch takes the scatter form (FP64 atomic sums) at every size. */
typedef struct lsq_batch_s *lsq_batch;

typedef struct {
  int64_t m, n;       /* size: m >= n >= 1, n <= the batch's n_max */
  const double *A;    /* device: m x n row-major (lda = n) */
  const double *b;    /* device: m */
  double *x;          /* device: n, the solution (written) */
  uint64_t seed;      /* Philox key of the item's sketch */
  int32_t method;     /* 0: FOSSILS, 1: SPIR */
  int32_t status;     /* written: the item's lsq_status */
} lsq_batch_item;

/* Workspace for batches of up to max_items (<= 256) problems with n <= n_max (<= 256)
 * and sum over items of m * ceil4(n) <= elems_max (the items' FP32 planes),
 * on the current device, working on cuda_stream (cudaStream_t; NULL: a
 * stream of its own).  The row-parallel passes take 1, 2 or 4 CTAs per SM,
 * chosen by timing the batch's residual pass the first time a shape class
 * (item count and total m n, in powers of two) is seen; the choices are kept
 * for the process and, when the environment variable LSQ_AUTOTUNE_FILE names
 * a file, appended to it and read back by later processes.
 * Errors: LSQ_ERR_INVALID, LSQ_ERR_OOM, LSQ_ERR_CUDA. */
lsq_status lsq_batch_create(int max_items, int64_t n_max, int64_t elems_max, void *cuda_stream,
                            lsq_batch *out);

/* Solve count items (1 <= count <= max_items); returns after every x is
 * written.  items[i].status gets each item's status (LSQ_OK,
 * LSQ_WARN_RANK_DEFICIENT, LSQ_ERR_NONFINITE, LSQ_ERR_INVALID for a zero
 * column); infos (count entries, may be NULL) the per-item counts,
 * condest and ||c_i||.  Returns the first error among the items, else
 * LSQ_OK; LSQ_ERR_INVALID for bad arguments (nothing run). */
lsq_status lsq_batch_solve(lsq_batch batch, int count, lsq_batch_item *items, lsq_info *infos);

/* Free the workspace.  NULL is ignored. */
void lsq_batch_destroy(lsq_batch batch);

/* ---- served stream: continuous batching of independent solves ---------- */

typedef struct lsq_server_s *lsq_server;

/* Create a request server on the current device.  arena_bytes of device
 * memory hold the admitted requests' A, b and x; max_slots solves run at
 * once, each on its own stream with a plan sized for m_max x n_max (plus that
 * plan's workspace, outside the arena).  The paper has no serving layer
 * (its solvers are one-shot); this is the library's own.
 * Errors: LSQ_ERR_INVALID (1 <= max_slots <= 64, n_max <= LSQ_MAX_N),
 * LSQ_ERR_OOM, LSQ_ERR_CUDA. */
lsq_status lsq_server_create(size_t arena_bytes, int max_slots, int64_t m_max, int64_t n_max,
                             lsq_server *out);

/* As lsq_server_create, but the requests are solved in lockstep batches
 * (lsq_batch_solve): each of `workers` worker threads owns a batch engine
 * for up to max_batch (<= 256) problems with n <= n_max (<= 256) and takes, first
 * come first served, as many queued requests as its batch, its planes and
 * the arena admit; requests that arrive while batches run wait for the next
 * free worker.  FOSSILS and SPIR only (method 0 or 1).  Device memory: the
 * arena plus, per worker, FP32 planes of min(arena_bytes / 8,
 * max_batch m_max n_max) entries (8 bytes each; at least m_max n_max).
 * Errors: LSQ_ERR_INVALID, LSQ_ERR_OOM, LSQ_ERR_CUDA. */
lsq_status lsq_server_create_batched(size_t arena_bytes, int workers, int max_batch,
                                     int64_t m_max, int64_t n_max, lsq_server *out);

/* Submit one FOSSILS (method 0), SPIR (method 1) or LSQR-based SPIR
 * (method 2) solve; returns at once
 * with a ticket.  opt: m <= m_max, n <= n_max, lda = n (or 0), zeta <= 8,
 * FP64 precision, one right-hand side; the other options as for a plan.
 * A (m x n row-major) and b (m) are host (on_device = 0) or device pointers;
 * they are copied into the arena when the request is admitted (first come,
 * first served, once a slot and its footprint 8(mn + m + n) bytes are free),
 * so they must stay valid and unchanged until lsq_poll stops returning
 * LSQ_PENDING.  Device inputs are copied on the server's own streams, which
 * are not ordered after any stream of the caller: the work that produced A
 * and b must be complete (its stream synchronized) before lsq_submit.  Errors: LSQ_ERR_INVALID; LSQ_ERR_OOM when the footprint can
 * never fit the arena (refused at admission time, nothing queued). */
lsq_status lsq_submit(lsq_server srv, const lsq_options *opt, int method, const double *A,
                      const double *b, int on_device, uint64_t *ticket);

/* LSQ_PENDING while the request is queued or running.  Once done: copies x
 * (n doubles) to the HOST buffer x (may be NULL), the solve's lsq_info to
 * info (may be NULL) and the submit-to-completion time in seconds to
 * latency_s (may be NULL), forgets the ticket and returns the solve's status. */
lsq_status lsq_poll(lsq_server srv, uint64_t ticket, double *x, lsq_info *info,
                    double *latency_s);

/* Counters: out7 = {submitted, completed, queued, running, arena bytes,
 * arena bytes in use, peak arena bytes in use}. */
lsq_status lsq_server_stats(lsq_server srv, int64_t *out7);

/* Stop the workers after their current solves and free everything; tickets
 * not polled yet are dropped.  NULL is ignored. */
void lsq_server_destroy(lsq_server srv);

/* Message for the last error on the calling thread ("" if none). */
const char *lsq_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LSQ_H */

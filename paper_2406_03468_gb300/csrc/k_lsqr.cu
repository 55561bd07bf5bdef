// LSQR-based SPIR (Sec. 4.2, "SPIR: conjugate gradient or LSQR?"): each
// refinement step's least-squares problem min || r_i - B dy ||, with
// B = A D^{-1} R^{-1} (column scaling and the sketch's R as a right
// preconditioner, eq. (ls-itref)), solved by LSQR (Paige and Saunders) from
// dy = 0, with SPIR's two stopping rules applied to the LSQR step
// (phi_k / rho_k) w_k.
//
// Golub-Kahan bidiagonalisation needs B v and B^T u per iteration.  Both come
// from ONE pass over A: with q_{k+1} = B v_k - alpha_k u_k (unnormalised,
// u_k = q_k / beta_k), the row i of q_{k+1} is (a_i . z) - (alpha_k /
// beta_k) q_k[i] with z = D^{-1} R^{-1} v_k, and row i's share of
// A^T q_{k+1} is a_i q_{k+1}[i] -- known as soon as the row's q is.  So the
// pass is shaped like the residual pass: the m-vector s holds -q_k, the pass
// computes r = bscale s - A z (= -q_{k+1}, with bscale = alpha_k / beta_k in
// the sign convention below), writes it back to s, and sums A^T r and
// ||r||^2 = beta_{k+1}^2.  The n-vector recurrences run on one CTA.
//
// Sign convention: s starts as r_i = q_1 (written by the step's FP64
// residual pass), so the first pass takes bscale = +alpha_1 / beta_1; every
// pass leaves s = -q_{k+1}, so later passes take bscale = -alpha_k / beta_k.
// R^{-T} D^{-1} A^T s is then -B^T q_{k+1}.
//
// Two forms of the pass: lsqr_df_kernel below, on the hi / lo FP32 planes of
// A in double-float (the default, as the inner passes of FOSSILS and SPIR),
// and the FP64 residual pass of k_pass.cu with bscale and s (two FP64 FMAs per
// element; inner_fp64_fma = 1 or planes out of range).
#include "lsq_common.cuh"
#include "lsq_dev.cuh"

namespace lsq {

namespace {

constexpr int kLqStages = 2;
constexpr int kLqFlush = 32;
constexpr uint64_t kLqWaitNs = 1000ull * 1000 * 1000;  // 1 s per TMA wait

template <int NC>
__device__ __forceinline__ void lq_load_vec(const double *__restrict__ x, int n, int lane,
                                            double (&v)[2 * NC]) {
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    v[2 * k] = (col < n) ? x[col] : 0.0;
    v[2 * k + 1] = (col + 1 < n) ? x[col + 1] : 0.0;
  }
}

// r = (*bscale) s - A z (row products in double-float on the planes, the row
// result and r in FP64), s <- r, partial sums of A^T r (double-float column
// sums flushed into FP64 every kLqFlush rows) and of ||r||^2 (FP64).  Rows
// are staged by TMA bulk copies (kLqStages per warp), waits bounded.
template <int NC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    lsqr_df_kernel(const float *__restrict__ Ahi, const float *__restrict__ Alo, int64_t ld32,
                   int64_t m, int n, const double *__restrict__ z, double *s,
                   const double *bscale, double *__restrict__ part, double *__restrict__ r2part,
                   int npad, const DevState *gate, int *err) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  extern __shared__ __align__(16) double lacc[];
  __shared__ double wmax[kPassThreads / 32];
  __shared__ double wr2[kPassThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float *stages = reinterpret_cast<float *>(lacc + (size_t)nw * NC * 64);
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)nw * kLqStages * 2 * NC * 64);
  float *wst = stages + (size_t)warp * kLqStages * 2 * NC * 64;
  uint64_t *wbar = bars + warp * kLqStages;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  const int64_t nrows = (r1 - r0 - warp + nw - 1) / nw > 0 ? (r1 - r0 - warp + nw - 1) / nw : 0;
  const unsigned row_bytes = (unsigned)(ld32 * sizeof(float));
  if (lane == 0) {
    for (int st = 0; st < kLqStages; st++) mbar_init(wbar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t pol = l2_evict_first();
  auto issue = [&](int64_t q) {
    if (lane == 0 && q < nrows) {
      const int64_t i = r0 + warp + q * nw;
      const int stg = (int)(q % kLqStages);
      float *dh = wst + (size_t)stg * 2 * NC * 64;
      mbar_expect_tx(wbar + stg, 2 * row_bytes);
      bulk_g2s(dh, Ahi + i * ld32, row_bytes, wbar + stg, pol);
      bulk_g2s(dh + NC * 64, Alo + i * ld32, row_bytes, wbar + stg, pol);
    }
  };
  for (int64_t q = 0; q < kLqStages; q++) issue(q);

  double *hw = lacc + (size_t)warp * NC * 64;
  for (int i = lane; i < NC * 64; i += 32) hw[i] = 0.0;
  double zr[2 * NC];
  lq_load_vec<NC>(z, n, lane, zr);
  double zmax = 0.0;
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) zmax = fmax(zmax, fabs(zr[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
  if (lane == 0) wmax[warp] = zmax;
  __syncthreads();
  zmax = 0.0;
  for (int w = 0; w < nw; w++) zmax = fmax(zmax, wmax[w]);
  int fz = 0;
  if (zmax > 0.0) frexp(zmax, &fz);
  // work in units of 2^fz: z' = z 2^-fz, r' = r 2^-fz (exact scalings)
  const double down = ldexp(1.0, -fz), up = ldexp(1.0, fz);
  const double bs = *bscale * down;
  f2_t zh[NC], zl[NC], zn[NC], hh[NC], hl[NC];
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const double v0 = zr[2 * k] * down, v1 = zr[2 * k + 1] * down;
    const float h0 = __double2float_rn(v0), h1 = __double2float_rn(v1);
    zh[k] = f2_pack(h0, h1);
    zl[k] = f2_pack(__double2float_rn(v0 - (double)h0), __double2float_rn(v1 - (double)h1));
    zn[k] = f2_pack(-h0, -h1);
    hh[k] = hl[k] = 0ull;
  }
  double r2 = 0.0;
  int blk = 0;
  int64_t qfail = -1;
  for (int64_t q = 0; q < nrows; q++) {
    const int stg = (int)(q % kLqStages);
    if (!__all_sync(0xffffffffu, mbar_wait(wbar + stg, (unsigned)((q / kLqStages) & 1), kLqWaitNs))) {
      qfail = q;
      break;
    }
    const int64_t i = r0 + warp + q * nw;
    const float *rh = wst + (size_t)stg * 2 * NC * 64;
    const float *rl = rh + NC * 64;
    f2_t ah[NC], al[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) {
      const int col = 64 * k + 2 * lane;
      if (col + 1 < n) {
        ah[k] = *reinterpret_cast<const f2_t *>(rh + col);
        al[k] = *reinterpret_cast<const f2_t *>(rl + col);
      } else {
        ah[k] = (col < n) ? f2_pack(rh[col], 0.0f) : 0ull;
        al[k] = (col < n) ? f2_pack(rl[col], 0.0f) : 0ull;
      }
    }
    const double si = s[i];
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(q + kLqStages);
    // row product t' = a_i . z' in double-float
    f2_t shp = 0ull, slp = 0ull;
#pragma unroll
    for (int k = 0; k < NC; k++) f2_dd_step(shp, slp, ah[k], al[k], zh[k], zl[k], zn[k]);
    float sh_, sl_;
    {
      float er;
      two_sum_f(f2_lo(shp), f2_hi(shp), sh_, er);
      sl_ = __fadd_rn(__fadd_rn(f2_lo(slp), f2_hi(slp)), er);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, sh_, o);
      const float ol = __shfl_xor_sync(0xffffffffu, sl_, o);
      float sm, er;
      two_sum_f(sh_, oh, sm, er);
      sh_ = sm;
      sl_ = __fadd_rn(__fadd_rn(sl_, ol), er);
    }
    // r' = bs s_i - t' in FP64; s_i <- r = r' 2^fz
    const double rp = fma(bs, si, -(widen(sh_) + widen(sl_)));
    if (lane == 0) {
      s[i] = rp * up;
      r2 = fma(rp, rp, r2);
    }
    // column sums h' += a_i r' (double-float)
    const float th = __double2float_rn(rp);
    const float tl = __double2float_rn(rp - (double)th);
    const f2_t th2 = f2_pack(th, th), tl2 = f2_pack(tl, tl), tn2 = f2_pack(-th, -th);
#pragma unroll
    for (int k = 0; k < NC; k++) f2_dd_step(hh[k], hl[k], ah[k], al[k], th2, tl2, tn2);
    if (++blk == kLqFlush) {
      blk = 0;
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        hw[col] += widen(f2_lo(hh[k])) + widen(f2_lo(hl[k]));
        hw[col + 1] += widen(f2_hi(hh[k])) + widen(f2_hi(hl[k]));
        hh[k] = hl[k] = 0ull;
      }
    }
  }
  if (qfail >= 0) {
    if (lane == 0) {
      if (err != nullptr) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      for (int64_t r = qfail; r < qfail + kLqStages && r < nrows; r++)
        mbar_wait(wbar + (r % kLqStages), (unsigned)((r / kLqStages) & 1), kLqWaitNs);
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    hw[col] += widen(f2_lo(hh[k])) + widen(f2_lo(hl[k]));
    hw[col + 1] += widen(f2_hi(hh[k])) + widen(f2_hi(hl[k]));
  }
  if (lane == 0) wr2[warp] = r2;
  __syncthreads();
  // fixed-order sums over the warps, scaled back: A^T r = 2^fz A^T r',
  // ||r||^2 = 2^(2 fz) ||r'||^2
  for (int c = threadIdx.x; c < npad; c += blockDim.x) {
    double sacc = 0.0;
    for (int w = 0; w < nw; w++) sacc += lacc[(size_t)w * NC * 64 + c];
    part[(size_t)blockIdx.x * npad + c] = sacc * up;
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; w++) t += wr2[w];
    r2part[blockIdx.x] = t * up * up;
  }
}

// LSQR start (Paige and Saunders' initialisation) from the step's right-hand
// side: beta_1 u_1 = r_i (kept in s by the residual pass), c = R^{-T} D^{-1}
// A^T r_i = beta_1 B^T u_1, so alpha_1 = ||c|| / beta_1, v_1 = c / ||c||,
// w_1 = v_1, phibar = beta_1, rhobar = alpha_1, dy = 0.
__global__ void __launch_bounds__(kVecThreads)
    lsqr_init_kernel(int n, const double *__restrict__ c, int step, double *v, double *w,
                     double *dy, int max_iters, int use_thresh, DevState *st) {
  const double beta = sqrt(st->r2);
  const double cn = sqrt(st->cnorm2[step]);
  const bool live = beta > 0.0 && cn > 0.0;
  const double inv = live ? 1.0 / cn : 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double vi = c[i] * inv;
    v[i] = vi;
    w[i] = vi;
    dy[i] = 0.0;
  }
  if (threadIdx.x == 0) {
    const double alpha = live ? cn / beta : 0.0;
    st->lq_alpha = alpha;
    st->lq_beta = beta;
    st->lq_phibar = beta;
    st->lq_rhobar = alpha;
    st->lq_bscale = live ? alpha / beta : 0.0;
    st->iters = 0;
    st->max_iters = max_iters;
    st->use_thresh = use_thresh;
    st->dnorm2 = 0.0;
    st->done = (max_iters <= 0 || !live) ? 1 : 0;
  }
}

// One LSQR iteration after the pass: p = R^{-T} D^{-1} A^T s = -B^T q_{k+1},
// beta_{k+1}^2 = st->lq_b2.  v <- (B^T u_{k+1} - beta v) / alpha, the plane
// rotation, dy += (phi / rho) w, w <- v - (theta / rho) w, and the stop test
// of SPIR's rules on the step (phi / rho) w.
__global__ void __launch_bounds__(kVecThreads)
    lsqr_update_kernel(int n, const double *__restrict__ p, double *v, double *w, double *dy,
                       DevState *st) {
  if (*(volatile int *)&st->done) return;
  __shared__ double scratch[32];
  const double beta = sqrt(st->lq_b2);
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
  double aa = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double vi = -p[i] * ib - beta * v[i];
    v[i] = vi;
    aa = fma(vi, vi, aa);
  }
  aa = block_sum(aa, scratch);
  const double alpha = sqrt(aa);
  const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
  const double rhobar = st->lq_rhobar, phibar = st->lq_phibar;
  const double rho = hypot(rhobar, beta);
  const double cs = rhobar / rho, sn = beta / rho;
  const double theta = sn * alpha;
  const double phi = cs * phibar;
  const double tstep = phi / rho, tw = theta / rho;
  double ss = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double vi = v[i] * ia;
    v[i] = vi;
    const double step = tstep * w[i];
    dy[i] += step;
    w[i] = vi - tw * w[i];
    ss = fma(step, step, ss);
  }
  ss = block_sum(ss, scratch);
  if (threadIdx.x == 0) {
    st->lq_alpha = alpha;
    st->lq_beta = beta;
    st->lq_rhobar = -cs * alpha;
    st->lq_phibar = sn * phibar;
    st->lq_bscale = beta > 0.0 ? -alpha / beta : 0.0;
    const int it = st->iters + 1;
    st->iters = it;
    st->dnorm2 = ss;
    bool stop = it >= st->max_iters || !(alpha > 0.0) || !(sn * phibar != 0.0);
    if (st->use_thresh && sqrt(ss) <= st->thresh1) stop = true;
    if (stop) st->done = 1;
  }
}

}  // namespace

cudaError_t launch_pass_lsqr_df(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                                const double *z, double *s, const double *bscale, double *part,
                                double *r2part, int grid, int npad, const DevState *gate, int *err,
                                cudaStream_t st) {
  const int nw = kPassThreads / 32;
  const size_t smem = (size_t)nw * npad * sizeof(double) +
                      (size_t)nw * kLqStages * 2 * npad * sizeof(float) +
                      (size_t)nw * kLqStages * sizeof(uint64_t);
  switch (npad / 64) {
#define LSQ_LQ_CASE(NCV)                                                                      \
  case NCV: {                                                                                 \
    if (smem > 48 * 1024) {                                                                   \
      cudaError_t e = ensure_smem_attr((const void *)lsqr_df_kernel<NCV>, (int)smem);         \
      if (e != cudaSuccess) return e;                                                         \
    }                                                                                         \
    lsqr_df_kernel<NCV><<<grid, kPassThreads, smem, st>>>(Ahi, Alo, ld32, m, n, z, s, bscale,   \
                                                          part, r2part, npad, gate, err);     \
    break;                                                                                    \
  }
    LSQ_LQ_CASE(1)
    LSQ_LQ_CASE(2)
    LSQ_LQ_CASE(4)
    LSQ_LQ_CASE(8)
    LSQ_LQ_CASE(16)
#undef LSQ_LQ_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_lsqr_init(int n, const double *c, int step, double *v, double *w, double *dy,
                             int max_iters, int use_thresh, DevState *st, cudaStream_t s) {
  lsqr_init_kernel<<<1, kVecThreads, 0, s>>>(n, c, step, v, w, dy, max_iters, use_thresh, st);
  return cudaGetLastError();
}

cudaError_t launch_lsqr_update(int n, const double *p, double *v, double *w, double *dy,
                               DevState *st, cudaStream_t s) {
  lsqr_update_kernel<<<1, kVecThreads, 0, s>>>(n, p, v, w, dy, st);
  return cudaGetLastError();
}

}  // namespace lsq

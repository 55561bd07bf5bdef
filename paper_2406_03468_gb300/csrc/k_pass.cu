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
#include "lsq_dev.cuh"

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

// ---------------------------------------------------------------------------
// Inner pass with the row dot products on the FP32 pipe.
//
// GB300 runs FP64 at about 2 FMA / clock / SM, so two FP64 FMAs per element
// (t_i += a_ij z_j and h_j += a_ij t_i) cap the pass near 30% of HBM.  Here
// t_i is evaluated exactly enough without FP64 arithmetic:
//   * a_ij (FP64, times 2^-Eg) is split into two FP32 words with integer
//     operations: hi = the leading 24 significant bits (exact), lo = the
//     remaining 29 bits rounded to FP32, so |a - hi - lo| <= 2^-48 |a|;
//   * z_j (times 2^Eg 2^-Fz, Fz from max |z'|) is split hi/lo by rounding;
//   * products hi*hi are exact as a pair (TwoProd with fmaf), the cross
//     terms hi*lo + lo*hi are added to the pair's error word, and the pairs
//     are summed with TwoSum (double-float accumulation), across the warp too;
//   * the resulting double-float t is converted to FP64 with integer
//     operations and one FP64 add.
// h_j += a_ij t_i stays a single FP64 FMA per element, so h keeps full FP64
// accumulation.  Power-of-two scalings are exact; h is scaled back by 2^Fz.
// The host takes this kernel only when every column norm is within 2^20 of
// the largest, which keeps every significant entry of A in FP32 range.
// ---------------------------------------------------------------------------

// a * 2^-Eg split into hi + lo (ebias = 896 + Eg).
__device__ __forceinline__ void split_f64(double a, int ebias, float &hi, float &lo) {
  const unsigned hw = (unsigned)__double2hiint(a), lw = (unsigned)__double2loint(a);
  const int ef = (int)((hw >> 20) & 0x7ffu) - ebias;
  const unsigned sign = hw & 0x80000000u;
  const unsigned hib = sign | ((unsigned)ef << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  const int lf = ef - 52;
  const float l = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __int_as_float((lf > 0 ? lf : 1) << 23));
  hi = (ef > 0) ? __uint_as_float(hib) : 0.0f;
  lo = (lf > 0) ? __uint_as_float(__float_as_uint(l) | sign) : 0.0f;
}

template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    atax_eft_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                    const double *__restrict__ z, int ebias, double zscale,
                    double *__restrict__ part, int npad, const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  __shared__ double sh[NC * 64];
  __shared__ double wmax[kPassThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  // z' = z * 2^Eg, then a common power of two 2^-Fz keeps z'' <= 1.
  double zr[2 * NC];
  load_vec<NC>(z, n, lane, zr);
  double zmax = 0.0;
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) {
    zr[k] *= zscale;
    zmax = fmax(zmax, fabs(zr[k]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zmax = fmax(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
  if (lane == 0) wmax[warp] = zmax;
  __syncthreads();
  zmax = 0.0;
  for (int w = 0; w < nw; w++) zmax = fmax(zmax, wmax[w]);
  int fz = 0;
  if (zmax > 0.0) frexp(zmax, &fz);
  const double down = ldexp(1.0, -fz), up = ldexp(1.0, fz);
  float zh[2 * NC], zl[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) {
    const double v = zr[k] * down;
    zh[k] = __double2float_rn(v);
    zl[k] = __double2float_rn(v - (double)zh[k]);
  }
  double h[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) h[k] = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    float sh_ = 0.0f, sl_ = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) {
      float ah, al;
      split_f64(a[k], ebias, ah, al);
      const float p = __fmul_rn(ah, zh[k]);
      const float e = __fmaf_rn(ah, zh[k], -p);
      const float c = __fmaf_rn(ah, zl[k], __fmaf_rn(al, zh[k], e));
      float s, err;
      two_sum_f(sh_, p, s, err);
      sh_ = s;
      sl_ = __fadd_rn(sl_, __fadd_rn(err, c));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, sh_, o);
      const float ol = __shfl_xor_sync(0xffffffffu, sl_, o);
      float s, err;
      two_sum_f(sh_, oh, s, err);
      sh_ = s;
      sl_ = __fadd_rn(__fadd_rn(sl_, ol), err);
    }
    const double t = widen(sh_) + widen(sl_);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) h[k] = fma(a[k], t, h[k]);
  }
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) h[k] *= up;
  cta_store_partial<NC>(h, sh, part, npad);
}

// ---------------------------------------------------------------------------
// Inner pass on the hi / lo FP32 planes of A (written by the sketch pass,
// a = hi + lo to 2^-48 |a|), all arithmetic on the FP32 pipe:
//   t_i = sum_j a_ij z_j : TwoProd of hi*z_hi, the cross terms hi*z_lo and
//         lo*z_hi added to the error word, TwoSum accumulation, double-float
//         warp reduction;
//   h_j += a_ij t_i      : the same products against t = t_hi + t_lo, each
//         column a double-float accumulator (TwoSum into the high word, the
//         error terms into the low word) flushed into an FP64 shared-memory
//         accumulator every kDfFlush = 32 rows of the warp.  A flush costs 32
//         FP64 warp instructions per warp (64 cycles each on its sub-
//         partition): every 8 rows it held the pass at 0.76 ms, every 32 rows
//         0.69 ms.  The low word then gathers up to 32 rows of error terms,
//         a worst-case relative error of about 2^-43 of the sums (2^-45 at 8
//         rows; every 128 rows, 2^-41, gained only 2% more).
// The FP64 pipe only sees the flushes (1/8 of an add per element), so the
// pass is no longer capped by GB300's FP64 rate.  z is scaled by a common
// power of two 2^-Fz; h is scaled back.
//
// Rows reach shared memory by TMA bulk copies (cp.async.bulk with mbarrier
// completion), kDfStages rows per warp in flight: lane 0 of each warp issues
// the copies of the rows its warp will process next while the warp computes
// on the current one, so the bytes in flight no longer depend on registers.
// Every mbarrier wait is bounded (kDfWaitNs); on a timeout the kernel
// records LSQ_ERR_TIMEOUT, waits (bounded) for its copies in flight and
// returns.
// ---------------------------------------------------------------------------
constexpr int kDfFlush = 32;
constexpr int kDfStages = 2;
constexpr uint64_t kDfWaitNs = 1000ull * 1000 * 1000;  // 1 s

template <int NC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    atax_df_kernel(const float *__restrict__ Ahi, const float *__restrict__ Alo, int64_t ld32,
                   int64_t m, int n, const double *__restrict__ z, double *__restrict__ part,
                   int npad, const DevState *gate, int *err, int64_t zstride,
                   int64_t pstride) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  // many right-hand sides: grid row blockIdx.y works on vector z_(blockIdx.y)
  z += (int64_t)blockIdx.y * zstride;
  part += (int64_t)blockIdx.y * pstride;
  // dynamic shared memory: [warps][NC*64] FP64 flush accumulators, then
  // [warps][kDfStages][2][NC*64] FP32 row stages (hi, lo), then the mbarriers
  extern __shared__ __align__(16) double hacc[];
  __shared__ double wmax[kPassThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float *stages = reinterpret_cast<float *>(hacc + (size_t)nw * NC * 64);
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)nw * kDfStages * 2 * NC * 64);
  float *wst = stages + (size_t)warp * kDfStages * 2 * NC * 64;
  uint64_t *wbar = bars + warp * kDfStages;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  const int64_t nrows = (r1 - r0 - warp + nw - 1) / nw > 0 ? (r1 - r0 - warp + nw - 1) / nw : 0;
  const unsigned row_bytes = (unsigned)(ld32 * sizeof(float));
  if (lane == 0) {
    for (int st = 0; st < kDfStages; st++) mbar_init(wbar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // lane 0: bulk copies of the warp's q-th row (hi and lo) into stage q % kDfStages
  const uint64_t pol = l2_evict_first();
  auto issue = [&](int64_t q) {
    if (lane == 0 && q < nrows) {
      const int64_t i = r0 + warp + q * nw;
      const int stg = (int)(q % kDfStages);
      float *dh = wst + (size_t)stg * 2 * NC * 64;
      mbar_expect_tx(wbar + stg, 2 * row_bytes);
      bulk_g2s(dh, Ahi + i * ld32, row_bytes, wbar + stg, pol);
      bulk_g2s(dh + NC * 64, Alo + i * ld32, row_bytes, wbar + stg, pol);
    }
  };
  for (int64_t q = 0; q < kDfStages; q++) issue(q);

  double *hw = hacc + (size_t)warp * NC * 64;
  for (int i = lane; i < NC * 64; i += 32) hw[i] = 0.0;
  double zr[2 * NC];
  load_vec<NC>(z, n, lane, zr);
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
  const double down = ldexp(1.0, -fz), up = ldexp(1.0, fz);
  // column pairs (2k, 2k + 1) of this lane: z hi / lo / -hi and the
  // double-float column sums, packed
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
  int blk = 0;
  int64_t qfail = -1;
  for (int64_t q = 0; q < nrows; q++) {
    const int stg = (int)(q % kDfStages);
    // one decision per warp: a lane whose wait ran out takes the whole warp
    // to the drain below
    if (!__all_sync(0xffffffffu, mbar_wait(wbar + stg, (unsigned)((q / kDfStages) & 1), kDfWaitNs))) {
      qfail = q;
      break;
    }
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
    // every lane has its values: the stage may be refilled (generic reads
    // before the async-proxy writes of the next copy)
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(q + kDfStages);
    // two independent double-float accumulators (even / odd column, the
    // halves of one packed pair) halve the dependent TwoSum chain
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
      float s, er;
      two_sum_f(sh_, oh, s, er);
      sh_ = s;
      sl_ = __fadd_rn(__fadd_rn(sl_, ol), er);
    }
    // renormalise t (Fast2Sum: |sh_| >= |sl_| after the sums above)
    const float th = __fadd_rn(sh_, sl_);
    const float tl = __fsub_rn(sl_, __fsub_rn(th, sh_));
    // column sums: TwoSum into the high word, error terms into the low word;
    // the low word only gathers kDfFlush rows of small terms before the FP64
    // flush, so it is not renormalised row by row
    const f2_t th2 = f2_pack(th, th), tl2 = f2_pack(tl, tl), tn2 = f2_pack(-th, -th);
#pragma unroll
    for (int k = 0; k < NC; k++) f2_dd_step(hh[k], hl[k], ah[k], al[k], th2, tl2, tn2);
    if (++blk == kDfFlush) {
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
    // record the error; let the copies this warp has in flight (rows qfail
    // .. qfail + kDfStages - 1, one per stage) land before the CTA's shared
    // memory is released (bounded again)
    if (lane == 0) {
      if (err != nullptr) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      for (int64_t r = qfail; r < qfail + kDfStages && r < nrows; r++)
        mbar_wait(wbar + (r % kDfStages), (unsigned)((r / kDfStages) & 1), kDfWaitNs);
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    hw[col] += widen(f2_lo(hh[k])) + widen(f2_lo(hl[k]));
    hw[col + 1] += widen(f2_hi(hh[k])) + widen(f2_hi(hl[k]));
  }
  __syncthreads();
  // fixed-order sum over the warps of this CTA, scaled back by 2^Fz
  for (int c = threadIdx.x; c < npad; c += blockDim.x) {
    double sacc = 0.0;
    for (int w = 0; w < nw; w++) sacc += hacc[(size_t)w * NC * 64 + c];
    part[(size_t)blockIdx.x * npad + c] = sacc * up;
  }
}

// ---------------------------------------------------------------------------
// FP32 inner pass of the mixed-precision tier (condest below the gate): reads
// the hi plane of A (A rounded to FP32, 4 bytes per element), FP32 row
// products, FP32 column sums flushed into FP64 accumulators every 32 rows
// (bounds the FP32 accumulation error at about 32 u_32 per block).  z is
// scaled by a common power of two so that it sits in FP32 range; h is scaled
// back.  Rows reach shared memory by TMA bulk copies, k32Stages rows per
// warp in flight (lane 0 issues the copies of the rows its warp will take
// next while the warp works on the current one), with the same bounded
// mbarrier waits and drain as the double-float pass.
// ---------------------------------------------------------------------------
constexpr int k32Stages = 4;

template <int NC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    atax32_kernel(const float *__restrict__ A32, int64_t ld32, int64_t m, int n,
                  const double *__restrict__ z, double *__restrict__ part, int npad,
                  const DevState *gate, int *err) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  // dynamic shared memory: [warps][k32Stages][NC*64] FP32 row stages, then
  // the mbarriers
  extern __shared__ __align__(16) float rst[];
  __shared__ double sh[NC * 64];
  __shared__ double wmax[kPassThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float *wst = rst + (size_t)warp * k32Stages * NC * 64;
  uint64_t *bars = reinterpret_cast<uint64_t *>(rst + (size_t)nw * k32Stages * NC * 64);
  uint64_t *wbar = bars + warp * k32Stages;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  const int64_t nrows = (r1 - r0 - warp + nw - 1) / nw > 0 ? (r1 - r0 - warp + nw - 1) / nw : 0;
  const unsigned row_bytes = (unsigned)(ld32 * sizeof(float));
  if (lane == 0) {
    for (int st = 0; st < k32Stages; st++) mbar_init(wbar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t pol = l2_evict_first();
  auto issue = [&](int64_t q) {
    if (lane == 0 && q < nrows) {
      const int64_t i = r0 + warp + q * nw;
      const int stg = (int)(q % k32Stages);
      mbar_expect_tx(wbar + stg, row_bytes);
      bulk_g2s(wst + (size_t)stg * NC * 64, A32 + i * ld32, row_bytes, wbar + stg, pol);
    }
  };
  for (int64_t q = 0; q < k32Stages; q++) issue(q);
  double zr[2 * NC];
  load_vec<NC>(z, n, lane, zr);
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
  const double down = ldexp(1.0, -fz), up = ldexp(1.0, fz);
  float zf[2 * NC], hf[2 * NC];
  double hd[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) {
    zf[k] = __double2float_rn(zr[k] * down);
    hf[k] = 0.0f;
    hd[k] = 0.0;
  }
  int blk = 0;
  int64_t qfail = -1;
  for (int64_t q = 0; q < nrows; q++) {
    const int stg = (int)(q % k32Stages);
    // one decision per warp: a lane whose wait ran out takes the whole warp
    // to the drain below
    if (!__all_sync(0xffffffffu, mbar_wait(wbar + stg, (unsigned)((q / k32Stages) & 1), kDfWaitNs))) {
      qfail = q;
      break;
    }
    const float *row = wst + (size_t)stg * NC * 64;
    float a[2 * NC];
#pragma unroll
    for (int k = 0; k < NC; k++) {
      const int col = 64 * k + 2 * lane;
      if (col + 1 < n) {
        const float2 v = *reinterpret_cast<const float2 *>(row + col);
        a[2 * k] = v.x;
        a[2 * k + 1] = v.y;
      } else {
        a[2 * k] = (col < n) ? row[col] : 0.0f;
        a[2 * k + 1] = 0.0f;
      }
    }
    // every lane has its values: the stage may be refilled
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    issue(q + k32Stages);
    float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
    for (int k = 0; k < NC; k++) {
      t0 = __fmaf_rn(a[2 * k], zf[2 * k], t0);
      t1 = __fmaf_rn(a[2 * k + 1], zf[2 * k + 1], t1);
    }
    float t = t0 + t1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) hf[k] = __fmaf_rn(a[k], t, hf[k]);
    if (++blk == 32) {
      blk = 0;
#pragma unroll
      for (int k = 0; k < 2 * NC; k++) {
        hd[k] += (double)hf[k];
        hf[k] = 0.0f;
      }
    }
  }
  if (qfail >= 0) {
    // record the error; let the copies this warp has in flight (rows qfail
    // .. qfail + k32Stages - 1, one per stage) land before the CTA's shared
    // memory is released
    if (lane == 0) {
      if (err != nullptr) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      for (int64_t r = qfail; r < qfail + k32Stages && r < nrows; r++)
        mbar_wait(wbar + (r % k32Stages), (unsigned)((r / k32Stages) & 1), kDfWaitNs);
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) hd[k] = (hd[k] + (double)hf[k]) * up;
  cta_store_partial<NC>(hd, sh, part, npad);
}

// With Ahi != NULL the pass also writes the hi / lo FP32 planes of A: this
// pass is bound by the FP64 pipe with HBM to spare, so the plane stores cost
// almost nothing here (the large-problem sketch leaves them to the first
// residual pass of a solve).
template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    resid_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                 const double *b, const double *__restrict__ x,
                 double *__restrict__ part, double *__restrict__ r2_part, int npad,
                 float *__restrict__ Ahi, float *__restrict__ Alo, int64_t ld32,
                 const DevState *gate, const double *bscale, double *rout) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  __shared__ double sh[NC * 64];
  const double bs = bscale != nullptr ? *bscale : 1.0;
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
    if (Ahi != nullptr) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        float h0, l0, h1, l1;
        split_rn(a[2 * k], h0, l0);
        split_rn(a[2 * k + 1], h1, l1);
        if (col + 1 < n) {
          __stcs(reinterpret_cast<float2 *>(Ahi + i * ld32 + col), make_float2(h0, h1));
          __stcs(reinterpret_cast<float2 *>(Alo + i * ld32 + col), make_float2(l0, l1));
        } else if (col < n) {
          __stcs(Ahi + i * ld32 + col, h0);
          __stcs(Alo + i * ld32 + col, l0);
        }
      }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) s = fma(a[k], xr[k], s);
    s = warp_sum(s);
    const double r = (bscale != nullptr ? bs * b[i] : b[i]) - s;
    if (rout != nullptr) {
      __syncwarp();  // every lane has read b[i] (rout may be b)
      if (lane == 0) rout[i] = r;
    }
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

// ---------------------------------------------------------------------------
// Compensated residual pass (the sketched Karlson-Walden test of Alg. 4's
// second refinement step): r = b - A x and g = A^T r with the compensated dot
// product Dot2 of Ogita, Rump and Oishi (TwoProd by fma, TwoSum, the error
// terms summed alongside), so r and g carry errors of order u |r| and
// u |A^T| |r| rather than the u |A| |x| of a plain FP64 residual, which sits
// at the u ||A||_F threshold of the test.  Per row the lanes' (sum, error)
// pairs are combined with TwoSum across the warp; r = r_hi + r_lo.  Per
// column each lane keeps a (sum, error) pair over its rows; the CTA writes
// both (part2: [grid][2][npad], sums then errors) and reduce_dot2 adds them
// with TwoSum in a fixed order.  About ten FP64 operations per element and
// product, against one.  With cs non-NULL the matrix is fl(A diag(cs)) (the
// column-scaled problem, formed element by element) and x is in its
// coordinates: Alg. 4 runs its test on the scaled problem, where the scaled
// iterate is exact rather than rounded by the change of coordinates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e) {
  s = a + b;
  const double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 8 ? 1 : kPassCtasPerSm)
    resid_dot2_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                      const double *__restrict__ b, const double *__restrict__ x,
                      const double *__restrict__ cs, double *__restrict__ part2,
                      double *__restrict__ r2_part, int npad) {
  __shared__ double sh[NC * 64];
  __shared__ double csh[NC * 64];
  __shared__ double r2sh[kPassThreads / 32];
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) csh[i] = (cs && i < n) ? cs[i] : 1.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  double xr[2 * NC], gs[2 * NC], gc[2 * NC];
  load_vec<NC>(x, n, lane, xr);
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) gs[k] = gc[k] = 0.0;
  double r2 = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    if (cs) {
#pragma unroll
      for (int k = 0; k < 2 * NC; k++) a[k] *= csh[64 * (k >> 1) + 2 * lane + (k & 1)];
    }
    // this lane's part of b_i - a_i . x (b_i on lane 0)
    double s = (lane == 0) ? b[i] : 0.0, c = 0.0;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) {
      const double p = -a[k] * xr[k];
      const double ep = fma(-a[k], xr[k], -p);
      double t, es;
      two_sum_d(s, p, t, es);
      s = t;
      c += ep + es;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double os = __shfl_xor_sync(0xffffffffu, s, o);
      const double oc = __shfl_xor_sync(0xffffffffu, c, o);
      double t, es;
      two_sum_d(s, os, t, es);
      s = t;
      c += oc + es;
    }
    double rh, rl;
    two_sum_d(s, c, rh, rl);
    r2 = fma(rh, rh, r2);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) {
      const double p = a[k] * rh;
      const double ep = fma(a[k], rh, -p);
      double t, es;
      two_sum_d(gs[k], p, t, es);
      gs[k] = t;
      gc[k] += ep + es + a[k] * rl;
    }
  }
  if (lane == 0) r2sh[warp] = r2;
  // the CTA's (sum, error) pairs: sums by TwoSum over the warps in order
  double *ps = part2 + (size_t)blockIdx.x * 2 * npad, *pc = ps + npad;
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) sh[i] = 0.0;
  __shared__ double shc[NC * 64];
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) shc[i] = 0.0;
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < 2 * NC; k++) {
        const int col = 64 * (k >> 1) + 2 * lane + (k & 1);
        double t, es;
        two_sum_d(sh[col], gs[k], t, es);
        sh[col] = t;
        shc[col] += gc[k] + es;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npad; i += blockDim.x) {
    ps[i] = sh[i];
    pc[i] = shc[i];
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; w++) t += r2sh[w];
    r2_part[blockIdx.x] = t;
  }
}

// out[j] = scale[j] (sum_g ps[g][j] + sum_g pc[g][j]) with the sums of the
// partials' sums by TwoSum (one thread per column, a fixed order); *r2 = the
// residual partials' sum.
__global__ void reduce_dot2_kernel(const double *__restrict__ part2, int grid, int npad, int n,
                                   const double *__restrict__ scale, double *__restrict__ out,
                                   const double *__restrict__ r2_part, double *r2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    double s = 0.0, c = 0.0;
    for (int g = 0; g < grid; g++) {
      double t, es;
      two_sum_d(s, part2[(size_t)g * 2 * npad + j], t, es);
      s = t;
      c += part2[(size_t)g * 2 * npad + npad + j] + es;
    }
    out[j] = scale ? scale[j] * (s + c) : s + c;
  }
  if (r2 != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    double t = 0.0;
    for (int g = 0; g < grid; g++) t += r2_part[g];
    *r2 = t;
  }
}

// out[c n + j] = scale[j] sum_g part[(c grid + g) npad + j] for c < batch
// (the partials of a batched pass, one block of grid x npad per vector).
__global__ void reduce_batched_kernel(const double *__restrict__ part, int grid, int npad, int n,
                                      int batch, const double *__restrict__ scale,
                                      double *__restrict__ out, const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * batch) return;
  const int c = (int)(idx / n), j = (int)(idx % n);
  const double *pc = part + (size_t)c * grid * npad + j;
  double s = 0.0;
  for (int g = 0; g < grid; g++) s += pc[(size_t)g * npad];
  out[idx] = scale ? scale[j] * s : s;
}

// out[j] = scale[j] sum_g part[g npad + j]; *r2 = sum_g r2_part[g] (CTA 0).
// One CTA per 32 columns: warp w sums the partials g = w, w + 8, ... of the
// lane's column, then warp 0 adds the 8 warp sums in order (a fixed order,
// so the result is deterministic).  A sub-partition issues one FP64 warp
// instruction per 64 cycles, so the partials of a column are spread over
// all four sub-partitions rather than summed by one thread.
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads)
    reduce_kernel(const double *__restrict__ part, int grid, int npad, int n,
                  const double *__restrict__ scale, double *__restrict__ out,
                  const double *__restrict__ r2_part, double *r2, const DevState *gate) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  __shared__ double red[kReduceThreads / 32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kReduceThreads / 32;
  const int j = blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0;
  if (j < n) {
    int g = warp;
    for (; g + nw < grid; g += 2 * nw) {
      s0 += part[(size_t)g * npad + j];
      s1 += part[(size_t)(g + nw) * npad + j];
    }
    if (g < grid) s0 += part[(size_t)g * npad + j];
  }
  red[warp][lane] = s0 + s1;
  __syncthreads();
  if (warp == 0 && j < n) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += red[w][lane];
    out[j] = scale ? scale[j] * s : s;
  }
  if (r2 != nullptr && blockIdx.x == 0) {
    __syncthreads();
    double t = 0.0;
    for (int g = threadIdx.x; g < grid; g += kReduceThreads) t += r2_part[g];
    t = warp_sum(t);
    if (lane == 0) red[warp][32] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < nw; w++) u += red[w][32];
      *r2 = u;
    }
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

cudaError_t launch_pass_atax_eft(const double *A, int64_t lda, int64_t m, int n, const double *z,
                                 int col_exp, double *part, int grid, int npad,
                                 const DevState *gate, cudaStream_t s) {
  const bool vec = vec_ok(A, lda);
  const int ebias = 896 + col_exp;
  const double zscale = ldexp(1.0, col_exp);
  LSQ_PASS_SWITCH(npad, {
    if (vec) atax_eft_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, z, ebias, zscale, part, npad, gate);
    else atax_eft_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, z, ebias, zscale, part, npad, gate);
  });
  return cudaGetLastError();
}

cudaError_t launch_pass_atax_df(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                                const double *z, double *part, int grid, int npad,
                                const DevState *gate, int *err, cudaStream_t s, int batch,
                                int64_t zstride, int64_t pstride) {
  const int nw = kPassThreads / 32;
  const size_t smem = (size_t)nw * npad * sizeof(double) +
                      (size_t)nw * kDfStages * 2 * npad * sizeof(float) +
                      (size_t)nw * kDfStages * sizeof(uint64_t);
  const dim3 g(grid, batch);
  LSQ_PASS_SWITCH(npad, {
    if (smem > 48 * 1024) {
      cudaError_t e = ensure_smem_attr((const void *)atax_df_kernel<NC>, (int)smem);
      if (e != cudaSuccess) return e;
    }
    atax_df_kernel<NC><<<g, kPassThreads, smem, s>>>(Ahi, Alo, ld32, m, n, z, part, npad, gate,
                                                     err, zstride, pstride);
  });
  return cudaGetLastError();
}

cudaError_t launch_pass_atax32(const float *A32, int64_t ld32, int64_t m, int n, const double *z,
                               double *part, int grid, int npad, const DevState *gate, int *err,
                               cudaStream_t s) {
  const int nw = kPassThreads / 32;
  const size_t smem = (size_t)nw * k32Stages * npad * sizeof(float) +
                      (size_t)nw * k32Stages * sizeof(uint64_t);
  LSQ_PASS_SWITCH(npad, {
    if (smem > 48 * 1024) {
      cudaError_t e = ensure_smem_attr((const void *)atax32_kernel<NC>, (int)smem);
      if (e != cudaSuccess) return e;
    }
    atax32_kernel<NC><<<grid, kPassThreads, smem, s>>>(A32, ld32, m, n, z, part, npad, gate, err);
  });
  return cudaGetLastError();
}

cudaError_t launch_pass_resid(const double *A, int64_t lda, int64_t m, int n, const double *b,
                              const double *x, double *part, double *r2_part, int grid, int npad,
                              cudaStream_t s, float *Ahi, float *Alo, int64_t ld32,
                              const DevState *gate, const double *bscale, double *rout) {
  const bool vec = vec_ok(A, lda);
  LSQ_PASS_SWITCH(npad, {
    if (vec)
      resid_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, part, r2_part,
                                                           npad, Ahi, Alo, ld32, gate, bscale,
                                                           rout);
    else
      resid_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, part, r2_part,
                                                            npad, Ahi, Alo, ld32, gate, bscale,
                                                            rout);
  });
  return cudaGetLastError();
}

cudaError_t launch_pass_resid_dot2(const double *A, int64_t lda, int64_t m, int n,
                                   const double *b, const double *x, const double *cs,
                                   double *part2, double *r2_part, int grid, int npad,
                                   cudaStream_t s) {
  const bool vec = vec_ok(A, lda);
  LSQ_PASS_SWITCH(npad, {
    if (vec)
      resid_dot2_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, cs, part2,
                                                                r2_part, npad);
    else
      resid_dot2_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, x, cs, part2,
                                                                 r2_part, npad);
  });
  return cudaGetLastError();
}

cudaError_t launch_reduce_dot2(const double *part2, int grid, int npad, int n, const double *scale,
                               double *out, const double *r2_part, double *r2, cudaStream_t s) {
  reduce_dot2_kernel<<<(n + 127) / 128, 128, 0, s>>>(part2, grid, npad, n, scale, out, r2_part, r2);
  return cudaGetLastError();
}

cudaError_t launch_reduce_batched(const double *part, int grid, int npad, int n, int batch,
                                  const double *scale, double *out, const DevState *gate,
                                  cudaStream_t s) {
  const int64_t cnt = (int64_t)n * batch;
  reduce_batched_kernel<<<(unsigned)((cnt + 127) / 128), 128, 0, s>>>(part, grid, npad, n, batch,
                                                                      scale, out, gate);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *part, int grid, int npad, int n, const double *scale,
                          double *out, const double *r2_part, double *r2, const DevState *gate,
                          cudaStream_t s) {
  reduce_kernel<<<(n + 31) / 32, kReduceThreads, 0, s>>>(part, grid, npad, n, scale, out, r2_part,
                                                       r2, gate);
  return cudaGetLastError();
}

}  // namespace lsq

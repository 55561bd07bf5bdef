// Inner pass for many right-hand sides: H = A^T (A Z) for up to 64 vectors
// z_c (Alg. 1's Apply, once per right-hand side, all sharing one sketch and
// one R) in ONE read of the hi / lo FP32 planes of A.
//
// The single-vector pass streams A once per vector; for k vectors that is k
// reads of A (64 x 3.2 GB per pass at 2e6 x 200).  Here each CTA stages a
// block of RB = 8 RPW rows by TMA bulk copy and applies it to all vectors while
// it sits in shared memory:
//   phase 1:  Y = A_blk Z        (RB x 64, double-float dot products)
//   phase 2:  H += A_blk^T Y     (n x 64 double-float accumulators in
//                                 registers, one tile per thread)
// so A leaves HBM once per pass and the work is FP32-pipe arithmetic: two
// double-float multiply-adds per element of A and per vector.
//
// Arithmetic is the single-vector double-float pass's (k_pass.cu): A =
// hi + lo exactly to 2^-48 |a|, each z_c split hi + lo after scaling by a
// power of two 2^-Fz_c (|z_c| < 1), products by TwoProd (fma) with the cross
// terms hi*lo + lo*hi added to the error word, sums by TwoSum.  Each
// (sum, error word) pair is renormalised by TwoSum every 32 terms of a dot
// product and after every row block of the column sums, and the column sums
// are added into FP64 every kMdFlushBlocks blocks, so no error word gathers
// more than 32 rounding errors of its own size.
//
// Layout: vector c of Z at Z + c n (n x k column-major), partial sums of CTA
// g for vector c at part + (c G + g) npad (the layout reduce_batched sums).
// Lane l works on vectors 2l and 2l + 1 (k is padded to 64 with zero
// vectors); in phase 1 warp w on rows RPW w .. RPW w + RPW - 1 of the block,
// in phase 2 on the column groups w, w + 8, w + 16, ... (4 columns each).
#include "lsq_common.cuh"
#include "lsq_dev.cuh"

namespace lsq {

namespace {

constexpr int kMdThreads = 256;
constexpr int kMdWarps = kMdThreads / 32;
constexpr int kMdVec = 64;            // vectors per launch: 2 per lane
constexpr int kMdFlushBlocks = 16;    // FP64 flush of the column sums
constexpr int kMdRenormJ = 32;        // dot-product terms between renormalisations
constexpr uint64_t kMdWaitNs = 1000ull * 1000 * 1000;  // 1 s per TMA wait

__device__ __forceinline__ f2_t f2_bcast(float v) { return f2_pack(v, v); }
__device__ __forceinline__ f2_t f2_neg(f2_t v) { return v ^ 0x8000000080000000ull; }

// Shared memory (dynamic, 16-byte aligned):
//   zs     [n4][32] float4  (zh_2l, zh_2l+1, zl_2l, zl_2l+1) per column j, lane l
//   ys     [RB][32] float4  the block's Y in the same pairing
//   stages [2][2][RB ld32]  float  hi plane rows, lo plane rows
//   bars   [2]      uint64
template <int RPW>
constexpr int md_rows() { return RPW * kMdWarps; }

size_t md_smem(int n, int64_t ld32, int rpw) {
  const size_t n4 = (size_t)(n + 3) / 4 * 4;
  const size_t rb = (size_t)rpw * kMdWarps;
  return n4 * 32 * 16 + rb * 32 * 16 + 4 * rb * (size_t)ld32 * sizeof(float) + 2 * sizeof(uint64_t);
}

template <int RPW, int JT4>
__global__ void __launch_bounds__(kMdThreads, 1)
    atax_df_multi_kernel(const float *__restrict__ Ahi, const float *__restrict__ Alo,
                         int64_t ld32, int64_t m, int n, const double *__restrict__ Z, int k,
                         double *__restrict__ part, int npad, const DevState *gate, int *err) {
  if (gate != nullptr && *(volatile const int *)&gate->done) return;
  constexpr int RB = md_rows<RPW>();
  extern __shared__ __align__(16) float4 msm4[];
  __shared__ int fz[kMdVec];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n4 = (n + 3) / 4 * 4;
  float4 *zs = msm4;
  float4 *ys = zs + (size_t)n4 * 32;
  float *stg = reinterpret_cast<float *>(ys + RB * 32);
  uint64_t *bars = reinterpret_cast<uint64_t *>(stg + 4 * (size_t)RB * ld32);
  const int G = gridDim.x;
  const int64_t per = (m + G - 1) / G;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  const int64_t nblk = (r1 - r0 + RB - 1) / RB;
  const uint64_t pol = l2_evict_first();
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: bulk copies of block q (hi and lo rows) into stage q & 1
  auto issue = [&](int64_t q) {
    if (q < nblk) {
      const int64_t i0 = r0 + q * RB;
      const int rows = (int)min((int64_t)RB, r1 - i0);
      const unsigned bytes = (unsigned)(rows * ld32 * sizeof(float));
      float *dh = stg + (size_t)(q & 1) * 2 * RB * ld32;
      mbar_expect_tx(bars + (q & 1), 2 * bytes);
      bulk_g2s(dh, Ahi + i0 * ld32, bytes, bars + (q & 1), pol);
      bulk_g2s(dh + (size_t)RB * ld32, Alo + i0 * ld32, bytes, bars + (q & 1), pol);
    }
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  // per-vector scale: max |z_c| < 2^fz[c]
  for (int c = warp; c < kMdVec; c += kMdWarps) {
    double mx = 0.0;
    if (c < k)
      for (int j = lane; j < n; j += 32) mx = fmax(mx, fabs(Z[(size_t)c * n + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      int e = 0;
      if (mx > 0.0) frexp(mx, &e);
      fz[c] = e;
    }
  }
  __syncthreads();
  // z split into hi / lo FP32 (zero for columns j >= n and vectors c >= k)
  for (int idx = tid; idx < n4 * 32; idx += kMdThreads) {
    const int j = idx >> 5, l = idx & 31, c0 = 2 * l, c1 = 2 * l + 1;
    const double v0 = (j < n && c0 < k) ? ldexp(Z[(size_t)c0 * n + j], -fz[c0]) : 0.0;
    const double v1 = (j < n && c1 < k) ? ldexp(Z[(size_t)c1 * n + j], -fz[c1]) : 0.0;
    const float h0 = __double2float_rn(v0), h1 = __double2float_rn(v1);
    zs[idx] = make_float4(h0, h1, __double2float_rn(v0 - (double)h0),
                          __double2float_rn(v1 - (double)h1));
  }
  __syncthreads();

  // phase-2 tile of this thread: columns 4 (warp + 8 g) .. + 3, g < JT4
  f2_t hh[4 * JT4], hl[4 * JT4];
#pragma unroll
  for (int t = 0; t < 4 * JT4; t++) hh[t] = hl[t] = 0ull;
  const int c0 = 2 * lane, c1 = 2 * lane + 1;
  const double sc0 = ldexp(1.0, fz[c0]), sc1 = ldexp(1.0, fz[c1]);
  bool first_flush = true;
  // H partial += the tile's double-float sums (scaled back); first flush stores
  auto flush = [&]() {
#pragma unroll
    for (int g = 0; g < JT4; g++) {
#pragma unroll
      for (int jj = 0; jj < 4; jj++) {
        const int j = 4 * (warp + kMdWarps * g) + jj;
        const int t = 4 * g + jj;
        if (j < n) {
          const double v0 = (widen(f2_lo(hh[t])) + widen(f2_lo(hl[t]))) * sc0;
          const double v1 = (widen(f2_hi(hh[t])) + widen(f2_hi(hl[t]))) * sc1;
          if (c0 < k) {
            double *p = part + ((size_t)c0 * G + blockIdx.x) * npad + j;
            *p = first_flush ? v0 : *p + v0;
          }
          if (c1 < k) {
            double *p = part + ((size_t)c1 * G + blockIdx.x) * npad + j;
            *p = first_flush ? v1 : *p + v1;
          }
        }
        hh[t] = hl[t] = 0ull;
      }
    }
    first_flush = false;
  };

  int64_t issued_hi = 1;  // thread 0: the last block issued (for the drain)
  bool ok = true;
  for (int64_t q = 0; q < nblk; q++) {
    const int st = (int)(q & 1);
    const bool landed = mbar_wait(bars + st, (unsigned)((q >> 1) & 1), kMdWaitNs);
    if (!__syncthreads_and(landed)) {
      ok = false;
      break;
    }
    const float *ah = stg + (size_t)st * 2 * RB * ld32;
    const float *al = ah + (size_t)RB * ld32;
    const int rows = (int)min((int64_t)RB, r1 - (r0 + q * RB));
    // ---- phase 1: y_i = a_i . z for the warp's rows, both lane vectors
    {
      f2_t s[RPW], l[RPW];
#pragma unroll
      for (int r = 0; r < RPW; r++) s[r] = l[r] = 0ull;
      for (int j4 = 0; j4 < n4; j4 += 4) {
        float4 a4h[RPW], a4l[RPW];
#pragma unroll
        for (int r = 0; r < RPW; r++) {
          const int i = RPW * warp + r;
          if (i < rows) {
            a4h[r] = *reinterpret_cast<const float4 *>(ah + (size_t)i * ld32 + j4);
            a4l[r] = *reinterpret_cast<const float4 *>(al + (size_t)i * ld32 + j4);
          } else {
            a4h[r] = a4l[r] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          // columns n .. n4 - 1 of the planes are padding: never read as data
          if (j4 + 4 > n) {
            if (j4 + 1 >= n) a4h[r].y = a4l[r].y = 0.f;
            if (j4 + 2 >= n) a4h[r].z = a4l[r].z = 0.f;
            if (j4 + 3 >= n) a4h[r].w = a4l[r].w = 0.f;
          }
        }
#pragma unroll
        for (int jj = 0; jj < 4; jj++) {
          const float4 z = zs[(size_t)(j4 + jj) * 32 + lane];
          const f2_t zh = f2_pack(z.x, z.y), zl = f2_pack(z.z, z.w), zn = f2_neg(zh);
#pragma unroll
          for (int r = 0; r < RPW; r++) {
            const float vh = jj == 0 ? a4h[r].x : jj == 1 ? a4h[r].y : jj == 2 ? a4h[r].z : a4h[r].w;
            const float vl = jj == 0 ? a4l[r].x : jj == 1 ? a4l[r].y : jj == 2 ? a4l[r].z : a4l[r].w;
            f2_dd_step(s[r], l[r], f2_bcast(vh), f2_bcast(vl), zh, zl, zn);
          }
        }
        if (((j4 + 4) % kMdRenormJ) == 0) {
#pragma unroll
          for (int r = 0; r < RPW; r++) f2_renorm(s[r], l[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < RPW; r++) {
        f2_renorm(s[r], l[r]);
        const int i = RPW * warp + r;
        ys[i * 32 + lane] = i < rows ? make_float4(f2_lo(s[r]), f2_hi(s[r]), f2_lo(l[r]), f2_hi(l[r]))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    // ---- phase 2: h_j += a_ij y_i over the block's rows, the thread's tile
    for (int i = 0; i < rows; i++) {
      const float4 y = ys[i * 32 + lane];
      const f2_t yh = f2_pack(y.x, y.y), yl = f2_pack(y.z, y.w), yn = f2_neg(yh);
      const float *rh = ah + (size_t)i * ld32, *rl = al + (size_t)i * ld32;
#pragma unroll
      for (int g = 0; g < JT4; g++) {
        const int j4 = 4 * (warp + kMdWarps * g);
        if (j4 < n) {
          float4 vh = *reinterpret_cast<const float4 *>(rh + j4);
          float4 vl = *reinterpret_cast<const float4 *>(rl + j4);
          if (j4 + 4 > n) {
            if (j4 + 1 >= n) vh.y = vl.y = 0.f;
            if (j4 + 2 >= n) vh.z = vl.z = 0.f;
            if (j4 + 3 >= n) vh.w = vl.w = 0.f;
          }
          f2_dd_step(hh[4 * g + 0], hl[4 * g + 0], f2_bcast(vh.x), f2_bcast(vl.x), yh, yl, yn);
          f2_dd_step(hh[4 * g + 1], hl[4 * g + 1], f2_bcast(vh.y), f2_bcast(vl.y), yh, yl, yn);
          f2_dd_step(hh[4 * g + 2], hl[4 * g + 2], f2_bcast(vh.z), f2_bcast(vl.z), yh, yl, yn);
          f2_dd_step(hh[4 * g + 3], hl[4 * g + 3], f2_bcast(vh.w), f2_bcast(vl.w), yh, yl, yn);
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 4 * JT4; t++) f2_renorm(hh[t], hl[t]);
    if ((q + 1) % kMdFlushBlocks == 0) flush();
    // every thread is done with stage st and with ys: order its generic reads
    // before the async-proxy writes of the refill, then refill the stage
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      issue(q + 2);
      if (q + 2 < nblk) issued_hi = q + 2;
    }
  }
  if (!ok) {
    // record the error; let the copies in flight land before the CTA's shared
    // memory is released (bounded again).  Blocks issued and not consumed:
    // at most one per stage, the last ones issued.
    if (tid == 0) {
      if (err != nullptr) atomicCAS(err, 0, (int)LSQ_ERR_TIMEOUT);
      for (int64_t q = issued_hi > 0 ? issued_hi - 1 : 0; q <= issued_hi && q < nblk; q++)
        mbar_wait(bars + (q & 1), (unsigned)((q >> 1) & 1), kMdWaitNs);
    }
    __syncthreads();
    return;
  }
  flush();  // the rest (and the stores of a CTA with fewer than kMdFlushBlocks blocks)
}

template <int RPW, int JT4>
cudaError_t launch_md(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                      const double *Z, int k, double *part, int grid, int npad,
                      const DevState *gate, int *err, cudaStream_t s) {
  const size_t smem = md_smem(n, ld32, RPW);
  const void *fn = (const void *)atax_df_multi_kernel<RPW, JT4>;
  cudaError_t e = ensure_smem_attr(fn, (int)smem);
  if (e != cudaSuccess) return e;
  atax_df_multi_kernel<RPW, JT4><<<grid, kMdThreads, smem, s>>>(Ahi, Alo, ld32, m, n, Z, k, part,
                                                                npad, gate, err);
  return cudaGetLastError();
}

template <int RPW>
cudaError_t launch_md_rpw(const float *Ahi, const float *Alo, int64_t ld32, int64_t m, int n,
                          const double *Z, int k, double *part, int grid, int npad,
                          const DevState *gate, int *err, cudaStream_t s) {
  // column groups of 4, dealt to the 8 warps in turn: JT4 = groups per warp
  const int jt4 = ((n + 3) / 4 + kMdWarps - 1) / kMdWarps;
  switch (jt4) {
    case 1: return launch_md<RPW, 1>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 2: return launch_md<RPW, 2>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 3: return launch_md<RPW, 3>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 4: return launch_md<RPW, 4>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 5: return launch_md<RPW, 5>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 6: return launch_md<RPW, 6>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 7: return launch_md<RPW, 7>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    case 8: return launch_md<RPW, 8>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Largest dynamic shared memory of one CTA (227 KB opt-in, minus the static part).
constexpr size_t kMdSmemMax = 225 * 1024;

bool multi_df_supported(int n, int k, int64_t ld32) {
  return n >= 1 && n <= 256 && k >= 1 && k <= kMdVec && ld32 % 4 == 0 &&
         md_smem(n, ld32, 2) <= kMdSmemMax;
}

cudaError_t launch_pass_atax_df_multi(const float *Ahi, const float *Alo, int64_t ld32, int64_t m,
                                      int n, const double *Z, int k, double *part, int grid,
                                      int npad, const DevState *gate, int *err, cudaStream_t s) {
  if (!multi_df_supported(n, k, ld32)) return cudaErrorInvalidValue;
  // four rows per warp in phase 1 when the stages fit (fewer shared-memory
  // loads of z per product), else two
  if (md_smem(n, ld32, 4) <= kMdSmemMax)
    return launch_md_rpw<4>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
  return launch_md_rpw<2>(Ahi, Alo, ld32, m, n, Z, k, part, grid, npad, gate, err, s);
}

}  // namespace lsq

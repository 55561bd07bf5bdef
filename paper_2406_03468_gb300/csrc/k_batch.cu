// Streaming passes of a batch of problems solved in lockstep (lsq_batch.cu):
// one launch covers every item, CTA g working on rows of item cta_item[g]
// (the CTAs are dealt to the items in proportion to their m n).  Per item the
// arithmetic is the single-problem passes' (k_pass.cu):
//   b_resid:  r = b - A x, partial sums of A^T r and ||r||^2, all FP64;
//   b_inner:  partial sums of A^T (A z) in double-float on the item's hi / lo
//             FP32 planes (TwoProd / TwoSum on packed f32x2 pairs, the column
//             sums flushed into FP64 every 32 rows), z scaled by a power of two;
//   b_reduce: the item's partials summed in a fixed order, times D^-1.
// n <= 256 (npad 64, 128 or 256).  The inner pass returns at once for an
// item whose inner loop has stopped (st->done), so the launch costs nothing
// for the items that are done.
#include "lsq_common.cuh"
#include "lsq_dev.cuh"

namespace lsq {

namespace {

constexpr int kBThreads = 256;
constexpr int kBFlush = 32;

template <int NC>
__device__ __forceinline__ void b_load_vec(const double *__restrict__ x, int n, int lane,
                                           double (&v)[2 * NC]) {
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    v[2 * k] = (col < n) ? x[col] : 0.0;
    v[2 * k + 1] = (col + 1 < n) ? x[col + 1] : 0.0;
  }
}

template <int NC>
__device__ __forceinline__ void b_load_row(const double *__restrict__ row, int n, int lane,
                                           double (&a)[2 * NC]) {
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    a[2 * k] = (col < n) ? __ldcs(row + col) : 0.0;
    a[2 * k + 1] = (col + 1 < n) ? __ldcs(row + col + 1) : 0.0;
  }
}

// Fixed-order sum over the CTA's warps of per-lane column values into
// part[0 .. npad).
template <int NC>
__device__ __forceinline__ void b_store_partial(const double (&h)[2 * NC], double *sh,
                                                double *__restrict__ part, int npad) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) sh[i] = 0.0;
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        sh[col] += h[2 * k];
        sh[col + 1] += h[2 * k + 1];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npad; i += blockDim.x) part[i] = sh[i];
}

template <int NC>
__device__ void b_resid_body(const BItem &it, int local, double *sh, double *r2sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = it.n;
  const int64_t m = it.m, per = (m + it.ncta - 1) / it.ncta;
  const int64_t r0 = min(m, (int64_t)local * per), r1 = min(m, r0 + per);
  double xr[2 * NC], g[2 * NC];
  b_load_vec<NC>(it.xo, n, lane, xr);
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) g[k] = 0.0;
  double r2 = 0.0;
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    b_load_row<NC>(it.A + i * n, n, lane, a);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) s = fma(a[k], xr[k], s);
    s = warp_sum(s);
    const double r = it.b[i] - s;
    r2 = fma(r, r, r2);
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) g[k] = fma(a[k], r, g[k]);
  }
  if (lane == 0) r2sh[warp] = r2;
  b_store_partial<NC>(g, sh, it.part + (size_t)local * it.npad, it.npad);
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += r2sh[w];
    it.r2part[local] = s;
  }
}

// The inner pass of one item's CTA: the structure of atax_df_kernel (the hi /
// lo planes staged by TMA bulk copies, kBStages per warp in flight, bounded
// mbarrier waits, drain on a timeout) over the item's row share.  A stage
// holds a block of consecutive rows, as many as fit in kBStageFloats floats
// per plane (16 rows at n = 32, 2 at n = 256), so that short rows still keep
// about 2 KB per plane and warp in flight; the warp takes its blocks in turn
// and the rows of a block one after the other.
// Shared memory: hacc [8 warps][256] FP64, stages [8][kBStages][2][512] FP32,
// then the mbarriers.
constexpr int kBStages = 2;
constexpr int kBStageFloats = 512;
constexpr uint64_t kBWaitNs = 1000ull * 1000 * 1000;  // 1 s
constexpr size_t kBInnerSmem =
    (size_t)(kBThreads / 32) * 256 * sizeof(double) +
    (size_t)(kBThreads / 32) * kBStages * 2 * kBStageFloats * sizeof(float) +
    (size_t)(kBThreads / 32) * kBStages * sizeof(uint64_t);

template <int NC>
__device__ void b_inner_body(const BItem &it, int local, double *hacc, double *wmax) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = it.n;
  const int64_t m = it.m, per = (m + it.ncta - 1) / it.ncta;
  const int64_t r0 = min(m, (int64_t)local * per), r1 = min(m, r0 + per);
  float *stages = reinterpret_cast<float *>(hacc + (size_t)nw * 256);
  uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)nw * kBStages * 2 * kBStageFloats);
  float *wst = stages + (size_t)warp * kBStages * 2 * kBStageFloats;
  uint64_t *wbar = bars + warp * kBStages;
  const int ld32 = it.ld32;
  const int rb = kBStageFloats / ld32;  // rows per block (ld32 <= 256: at least 2)
  const int64_t nblk_all = (r1 - r0 + rb - 1) / rb;
  const int64_t nblks = (nblk_all - warp + nw - 1) / nw > 0 ? (nblk_all - warp + nw - 1) / nw : 0;
  if (lane == 0) {
    for (int st = 0; st < kBStages; st++) mbar_init(wbar + st, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const uint64_t pol = l2_evict_first();
  // the warp's q-th block: rows r0 + (warp + q nw) rb .. (at most rb, within r1)
  auto block_rows = [&](int64_t q, int64_t &i0) {
    i0 = r0 + (warp + q * nw) * (int64_t)rb;
    return (int)min((int64_t)rb, r1 - i0);
  };
  auto issue = [&](int64_t q) {
    if (lane == 0 && q < nblks) {
      int64_t i0;
      const int rows = block_rows(q, i0);
      const unsigned bytes = (unsigned)(rows * ld32 * sizeof(float));
      const int stg = (int)(q % kBStages);
      float *dh = wst + (size_t)stg * 2 * kBStageFloats;
      mbar_expect_tx(wbar + stg, 2 * bytes);
      bulk_g2s(dh, it.Ahi + i0 * ld32, bytes, wbar + stg, pol);
      bulk_g2s(dh + kBStageFloats, it.Alo + i0 * ld32, bytes, wbar + stg, pol);
    }
  };
  for (int64_t q = 0; q < kBStages; q++) issue(q);
  double *hw = hacc + (size_t)warp * 256;
  for (int i = lane; i < NC * 64; i += 32) hw[i] = 0.0;
  double zr[2 * NC];
  b_load_vec<NC>(it.z, n, lane, zr);
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
  for (int64_t q = 0; q < nblks; q++) {
    const int stg = (int)(q % kBStages);
    if (!__all_sync(0xffffffffu, mbar_wait(wbar + stg, (unsigned)((q / kBStages) & 1), kBWaitNs))) {
      qfail = q;
      break;
    }
    int64_t i0;
    const int rows = block_rows(q, i0);
    for (int rr = 0; rr < rows; rr++) {
    const float *rh = wst + (size_t)stg * 2 * kBStageFloats + (size_t)rr * ld32;
    const float *rl = rh + kBStageFloats;
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
    if (rr == rows - 1) {
      // every lane has the block's values: the stage may be refilled
      __syncwarp();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(q + kBStages);
    }
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
    const float th = __fadd_rn(sh_, sl_);
    const float tl = __fsub_rn(sl_, __fsub_rn(th, sh_));
    const f2_t th2 = f2_pack(th, th), tl2 = f2_pack(tl, tl), tn2 = f2_pack(-th, -th);
#pragma unroll
    for (int k = 0; k < NC; k++) f2_dd_step(hh[k], hl[k], ah[k], al[k], th2, tl2, tn2);
    if (++blk == kBFlush) {
      blk = 0;
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        hw[col] += widen(f2_lo(hh[k])) + widen(f2_lo(hl[k]));
        hw[col + 1] += widen(f2_hi(hh[k])) + widen(f2_hi(hl[k]));
        hh[k] = hl[k] = 0ull;
      }
    }
    }  // rows of the block
  }
  if (qfail >= 0) {
    if (lane == 0) {
      atomicCAS(&it.st->err, 0, (int)LSQ_ERR_TIMEOUT);
      for (int64_t r = qfail; r < qfail + kBStages && r < nblks; r++)
        mbar_wait(wbar + (r % kBStages), (unsigned)((r / kBStages) & 1), kBWaitNs);
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
  double *part = it.part + (size_t)local * it.npad;
  for (int c = threadIdx.x; c < it.npad; c += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += hacc[(size_t)w * 256 + c];
    part[c] = s * up;
  }
}

__global__ void __launch_bounds__(kBThreads, 2)
    b_resid_kernel(const BItem *__restrict__ items, const int *__restrict__ cta_item) {
  __shared__ double sh[4 * 64];
  __shared__ double r2sh[kBThreads / 32];
  const int idx = cta_item[blockIdx.x];
  if (idx < 0) return;
  const BItem &it = items[idx];
  const int local = blockIdx.x - it.cta0;
  switch (it.npad / 64) {
    case 1: b_resid_body<1>(it, local, sh, r2sh); break;
    case 2: b_resid_body<2>(it, local, sh, r2sh); break;
    case 4: b_resid_body<4>(it, local, sh, r2sh); break;
    default: break;
  }
}

__global__ void __launch_bounds__(kBThreads, 2)
    b_inner_kernel(const BItem *__restrict__ items, const int *__restrict__ cta_item) {
  extern __shared__ __align__(16) double hacc[];
  __shared__ double wmax[kBThreads / 32];
  const int idx = cta_item[blockIdx.x];
  if (idx < 0) return;
  const BItem &it = items[idx];
  if (*(volatile const int *)&it.st->done) return;
  const int local = blockIdx.x - it.cta0;
  switch (it.npad / 64) {
    case 1: b_inner_body<1>(it, local, hacc, wmax); break;
    case 2: b_inner_body<2>(it, local, hacc, wmax); break;
    case 4: b_inner_body<4>(it, local, hacc, wmax); break;
    default: break;
  }
}

// out[j] = dinv[j] sum_g part[g npad + j] over the item's CTAs (8 warps per
// 32 columns, each summing every 8th partial, then one warp adds the 8 in
// order); mode 0 also *r2 = sum of the residual partials.  Grid (column
// blocks, items).
__global__ void __launch_bounds__(256)
    b_reduce_kernel(const BItem *__restrict__ items, int mode) {
  __shared__ double red[8][33];
  const BItem &it = items[blockIdx.y];
  if (mode == 1 && *(volatile const int *)&it.st->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  if (blockIdx.x * 32 >= it.n && !(mode == 0 && blockIdx.x == 0)) return;
  double s = 0.0;
  if (j < it.n)
    for (int g = warp; g < it.ncta; g += 8) s += it.part[(size_t)g * it.npad + j];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && j < it.n) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[w][lane];
    (mode == 0 ? it.g : it.h)[j] = it.dinv[j] * t;
  }
  if (mode == 0 && blockIdx.x == 0) {
    __syncthreads();
    double t = 0.0;
    for (int g = threadIdx.x; g < it.ncta; g += 256) t += it.r2part[g];
    t = warp_sum(t);
    if (lane == 0) red[warp][32] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int w = 0; w < 8; w++) u += red[w][32];
      it.st->r2 = u;
    }
  }
}

// Deal the `grid` CTAs of the row-parallel passes to the items in proportion
// to m n: every item (all = 1) or only the items whose inner loop is still
// running (all = 0), so that the last items of a batch get the whole GPU.
// Writes cta0 / ncta of the table and the CTA -> item map (-1: no item).
// One CTA; the deal is done by thread 0 in a fixed order.
__global__ void b_redeal_kernel(BItem *__restrict__ items, int count, int *__restrict__ cta_item,
                                int grid, int all) {
  __shared__ int cnt[1024];
  if (threadIdx.x == 0) {
    double tot = 0.0;
    int act = 0;
    for (int i = 0; i < count; i++) {
      const bool on = all || !*(volatile const int *)&items[i].st->done;
      cnt[i] = on ? 1 : 0;
      if (on) {
        tot += (double)items[i].m * items[i].n;
        act++;
      }
    }
    int used = act;
    if (act > 0 && grid > act) {
      const int left = grid - act;
      for (int i = 0; i < count; i++)
        if (cnt[i]) {
          const int f = (int)floor((double)items[i].m * items[i].n / tot * left);
          cnt[i] += f;
          used += f;
        }
      // the rest one at a time, in item order
      for (int i = 0; used < grid; i = (i + 1) % count)
        if (cnt[i]) {
          cnt[i]++;
          used++;
        }
    }
    int g = 0;
    for (int i = 0; i < count; i++) {
      items[i].cta0 = g;
      items[i].ncta = cnt[i];
      g += cnt[i];
    }
  }
  __syncthreads();
  for (int i = 0; i < count; i++) {
    const int c0 = items[i].cta0, c = items[i].ncta;
    for (int k = threadIdx.x; k < c; k += blockDim.x) cta_item[c0 + k] = i;
  }
  const int g = items[count - 1].cta0 + items[count - 1].ncta;
  for (int k = g + threadIdx.x; k < grid; k += blockDim.x) cta_item[k] = -1;
}

// Zero every item's sketch accumulator SAb (d x (n + 1)) before the scatter.
__global__ void b_zero_kernel(const BItem *__restrict__ items) {
  const BItem &it = items[blockIdx.y];
  const int64_t cnt = (int64_t)it.d * (it.n + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x)
    it.SAb[i] = 0.0;
}

}  // namespace

cudaError_t launch_b_redeal(BItem *items, int count, int *cta_item, int grid, int all,
                            cudaStream_t s) {
  if (count > 1024) return cudaErrorInvalidValue;
  b_redeal_kernel<<<1, 256, 0, s>>>(items, count, cta_item, grid, all);
  return cudaGetLastError();
}

cudaError_t launch_b_zero(const BItem *items, int count, cudaStream_t s) {
  b_zero_kernel<<<dim3(64, count), 256, 0, s>>>(items);
  return cudaGetLastError();
}

cudaError_t launch_b_resid(const BItem *items, const int *cta_item, int grid, cudaStream_t s) {
  b_resid_kernel<<<grid, kBThreads, 0, s>>>(items, cta_item);
  return cudaGetLastError();
}

cudaError_t prepare_b_inner() {
  return ensure_smem_attr((const void *)b_inner_kernel, (int)kBInnerSmem);
}

cudaError_t launch_b_inner(const BItem *items, const int *cta_item, int grid, cudaStream_t s) {
  b_inner_kernel<<<grid, kBThreads, kBInnerSmem, s>>>(items, cta_item);
  return cudaGetLastError();
}

cudaError_t launch_b_reduce(const BItem *items, int count, int nmax, int mode, cudaStream_t s) {
  b_reduce_kernel<<<dim3((nmax + 31) / 32, count), 256, 0, s>>>(items, mode);
  return cudaGetLastError();
}

}  // namespace lsq

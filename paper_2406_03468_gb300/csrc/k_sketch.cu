// Sparse sign embedding and the sketch pass S [A b] (Sec. 4.2, "Choice of
// embedding"; Alg. 1, first line).
//
// S = zeta^{-1/2} [s_1 ... s_m]: column j of S has zeta nonzeros +-1 at
// distinct rows.  The rows and signs follow this library's Philox4x64-10
// spec (counter (j, t, 0, 0), key (seed, 0); 32-bit halves of each block,
// low half first; the first half of block 0 carries the sign bits; the rest
// are candidate rows floor(u d / 2^32) accepted unless repeated).
//
// The pass reads each row of A once (one warp per row, 16-byte loads) and
// scatters +-a_j into the zeta rows of the row-major, L2-resident sketch
// with FP64 reductions performed in L2; it also accumulates the column sums
// of squares for the column scaling of Alg. 4.  The finalize kernel turns
// the sums into column norms, applies diag(d)^{-1} and zeta^{-1/2}, and
// transposes the sketch to the column-major layout the QR works on.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t hi0 = __umul64hi(kPhiloxM0, c[0]), lo0 = kPhiloxM0 * c[0];
    const uint64_t hi1 = __umul64hi(kPhiloxM1, c[2]), lo1 = kPhiloxM1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// The zeta rows h[0 .. zeta) (-1 past the ones drawn) and the sign word of
// column j of S (row j of A), by the spec above.
template <int ZM>
__device__ __forceinline__ void column_pattern(int64_t j, int d, int zeta, uint64_t seed,
                                               int (&h)[ZM], uint32_t &sb_out) {
  int cnt = 0;
  uint32_t sb = 0;
#pragma unroll
  for (int k = 0; k < ZM; k++) h[k] = -1;
  // Bounded: at most 1<<16 blocks (the expected count is < 20 even for d = zeta = 32).
  for (uint64_t t = 0; cnt < zeta && t < (1ull << 16); t++) {
    uint64_t c[4] = {(uint64_t)j, t, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const uint32_t u = (q & 1) ? (uint32_t)(c[q >> 1] >> 32) : (uint32_t)(c[q >> 1]);
      if (t == 0 && q == 0) {
        sb = u;
        continue;
      }
      if (cnt >= zeta) continue;
      const int hh = (int)(((uint64_t)u * (uint64_t)d) >> 32);
      bool dup = false;
#pragma unroll
      for (int k = 0; k < ZM; k++) dup |= (k < cnt && h[k] == hh);
      if (!dup) {
#pragma unroll
        for (int k = 0; k < ZM; k++)
          if (k == cnt) h[k] = hh;
        cnt++;
      }
    }
  }
  sb_out = sb;
}

// One thread per column j of S (row j of A).
__global__ void pattern_kernel(int64_t m, int d, int zeta, uint64_t seed, int32_t *rows,
                               uint32_t *signbits) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= m) return;
  int h[kMaxZeta];
  uint32_t sb = 0;
  column_pattern<kMaxZeta>(j, d, zeta, seed, h, sb);
  for (int k = 0; k < zeta; k++) rows[j * zeta + k] = h[k];
  signbits[j] = sb;
}

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


__device__ __forceinline__ double flip_sign(double a, bool neg) {
  return __longlong_as_double(__double_as_longlong(a) ^ (neg ? (long long)0x8000000000000000ull : 0ll));
}

template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    sketch_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                  const double *__restrict__ b, int d, int zeta, const int32_t *__restrict__ rows,
                  const uint32_t *__restrict__ signbits, double *__restrict__ SAb,
                  double *__restrict__ colsq_part, int npad, float *__restrict__ Ahi,
                  float *__restrict__ Alo, int64_t ld32) {
  __shared__ double acc[NC * 64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  const int ldsa = n + 1;
  double sq[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) sq[k] = 0.0;

  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    const int myh = (lane < zeta) ? rows[i * zeta + lane] : 0;
    const uint32_t sb = signbits[i];
    if (Ahi != nullptr) {  // hi / lo FP32 planes of the row, written as it streams
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
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) sq[k] = fma(a[k], a[k], sq[k]);
    if (b != nullptr && lane < zeta && (unsigned)myh < (unsigned)d) {
      atomicAdd(SAb + (size_t)myh * ldsa + n, flip_sign(b[i], (sb >> lane) & 1u));
    }
    for (int t = 0; t < zeta; t++) {
      const int h = __shfl_sync(0xffffffffu, myh, t);
      if ((unsigned)h >= (unsigned)d) continue;
      const bool neg = (sb >> t) & 1u;
      double *dst = SAb + (size_t)h * ldsa;
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        if (col < n) atomicAdd(dst + col, flip_sign(a[2 * k], neg));
        if (col + 1 < n) atomicAdd(dst + col + 1, flip_sign(a[2 * k + 1], neg));
      }
    }
  }
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) acc[i] = 0.0;
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        acc[col] += sq[2 * k];
        acc[col + 1] += sq[2 * k + 1];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npad; i += blockDim.x)
    colsq_part[(size_t)blockIdx.x * npad + i] = acc[i];
}

__global__ void colnorm_kernel(const double *__restrict__ part, int grid, int npad, int n,
                               int col_scale, double *dcol, double *dinv, DevState *st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int g = 0; g < grid; g++) s += part[(size_t)g * npad + j];
  const double nrm = sqrt(s);
  if (!isfinite(nrm)) atomicExch(&st->nonfinite, 1);
  if (col_scale && nrm == 0.0) atomicExch(&st->zero_col, 1);
  dcol[j] = nrm;  // the column norm, also when the scaling is off
  dinv[j] = col_scale ? 1.0 / nrm : 1.0;
}

// W[c * d + h] = SAb[h * (n+1) + c] * scale_c, scale_c = dinv_c zeta^{-1/2}
// (c < n) or zeta^{-1/2} (c == n).  32 x 32 tiles through shared memory.
__global__ void transpose_scale_kernel(const double *__restrict__ SAb, int n, int d,
                                       const double *__restrict__ dinv, double zinv,
                                       double *__restrict__ W, DevState *st) {
  __shared__ double tile[32][33];
  const int ncols = n + 1;
  const int c0 = blockIdx.x * 32, h0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int h = h0 + r, c = c0 + threadIdx.x;
    if (h < d && c < ncols) {
      const double v = SAb[(size_t)h * ncols + c];
      if (!isfinite(v)) atomicExch(&st->nonfinite, 1);
      tile[r][threadIdx.x] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, h = h0 + threadIdx.x;
    if (h < d && c < ncols) {
      const double sc = (c < n) ? dinv[c] * zinv : zinv;
      W[(size_t)c * d + h] = tile[threadIdx.x][r] * sc;
    }
  }
}

// ---------------------------------------------------------------------------
// Gather form of the sketch pass.  The scatter above pays one L2 FP64 atomic
// per element of A and target row (zeta per element); on GB300 those run at
// about 0.6 G/s and bound the pass.  The gather form inverts the
// pattern once per plan into source lists (CSR by sketch row h: the rows i
// of A with h among their zeta rows, sorted by i) and gives each sketch row
// to one warp, which walks its list and sums the +-rows of A in registers.
// The sums are 64-bit fixed point per column: every entry is truncated once
// to a multiple of 2^F_j, F_j = E_j + L - 63 (|A_ij| < 2^E_j, L = bits of the
// longest list), and added exactly, so the sketch is reproducible bit for
// bit whatever the order, and each entry of S[A b] is the exact sum of the
// truncated terms, rounded once to FP64 (error < 2^(L-62) max_i |A_ij| per
// term, 2^-51 max_i |A_ij| for lists under 2^11 entries, plus one final
// rounding).  All warps of one column chunk sweep A in row
// order together, so the zeta reads of a row mostly hit L2.
// ---------------------------------------------------------------------------

constexpr int kGatherWarps = 8;      // warps per CTA of the gather kernel
constexpr int kSortMax = 16384;      // longest source list sorted in shared memory

__global__ void tgt_count_kernel(const int32_t *__restrict__ rows, int64_t mz, int d, int *cnt) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= mz) return;
  const int h = rows[e];
  if ((unsigned)h < (unsigned)d) atomicAdd(cnt + h, 1);
}

// Exclusive scan of cnt into ptr (d + 1 entries), longest list into *lmax,
// cnt reset to 0 (it becomes the fill cursor).  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
    tgt_scan_kernel(int *cnt, int d, int64_t *ptr, int *lmax) {
  __shared__ int64_t part[1024];
  __shared__ int pmax[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int per = (d + nt - 1) / nt;
  const int h0 = min(d, t * per), h1 = min(d, h0 + per);
  int64_t sum = 0;
  int mx = 0;
  for (int h = h0; h < h1; h++) {
    sum += cnt[h];
    mx = max(mx, cnt[h]);
  }
  part[t] = sum;
  pmax[t] = mx;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {  // inclusive Hillis-Steele scan
    const int64_t v = (t >= off) ? part[t - off] : 0;
    const int w = (t >= off) ? pmax[t - off] : 0;
    __syncthreads();
    part[t] += v;
    pmax[t] = max(pmax[t], w);
    __syncthreads();
  }
  int64_t run = part[t] - sum;
  for (int h = h0; h < h1; h++) {
    ptr[h] = run;
    run += cnt[h];
    cnt[h] = 0;
  }
  if (t == nt - 1) {
    ptr[d] = part[t];
    *lmax = pmax[t];
  }
}

__global__ void tgt_fill_kernel(const int32_t *__restrict__ rows, const uint32_t *__restrict__ sb,
                                int64_t m, int zeta, int d, const int64_t *__restrict__ ptr,
                                int *cursor, uint32_t *src) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m * zeta) return;
  const int h = rows[e];
  if ((unsigned)h >= (unsigned)d) return;
  const int64_t i = e / zeta;
  const int t = (int)(e - i * zeta);
  const uint32_t neg = (sb[i] >> t) & 1u;
  const int64_t pos = ptr[h] + atomicAdd(cursor + h, 1);
  src[pos] = (uint32_t)i | (neg << 31);
}

// Sort each source list by row (bitonic, in shared memory); one CTA per list.
__global__ void __launch_bounds__(512)
    tgt_sort_kernel(const int64_t *__restrict__ ptr, uint32_t *src) {
  extern __shared__ uint32_t keys[];
  const int64_t p0 = ptr[blockIdx.x];
  const int len = (int)(ptr[blockIdx.x + 1] - p0);
  if (len <= 1 || len > kSortMax) return;
  int P = 1;
  while (P < len) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) keys[i] = (i < len) ? src[p0 + i] : 0x7fffffffu;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t a = keys[i], c = keys[l];
          const bool up = ((i & k) == 0);
          const bool gt = (a & 0x7fffffffu) > (c & 0x7fffffffu);
          if (gt == up) {
            keys[i] = c;
            keys[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) src[p0 + i] = keys[i];
}

__device__ __forceinline__ int biased_exp(double a) {
  return (int)(((unsigned)__double2hiint(a) >> 20) & 0x7ffu);
}

// One streaming pass over A (no sketch): column sums of squares (partials,
// CTA g's at colsq_part + g pstride), the largest biased exponent per column
// and of b (atomicMax into colexp[0..n) and colexp[bslot], zeroed first), and
// the hi / lo FP32 planes when Ahi != NULL.  accumulate = 1 adds the partials
// to those of earlier rows (A in row chunks).  npad = 64 NC columns from A.
template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads, NC >= 16 ? 1 : kPassCtasPerSm)
    prep_kernel(const double *__restrict__ A, int64_t lda, int64_t m, int n,
                const double *__restrict__ b, double *__restrict__ colsq_part, int npad,
                int pstride, int *colexp, int bslot, float *__restrict__ Ahi,
                float *__restrict__ Alo, int64_t ld32, int accumulate) {
  __shared__ double acc[NC * 64];
  __shared__ int emax[NC * 64 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per), r1 = min(m, r0 + per);
  for (int i = threadIdx.x; i <= NC * 64; i += blockDim.x) emax[i] = 0;
  double sq[2 * NC];
  int ex[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) {
    sq[k] = 0.0;
    ex[k] = 0;
  }
  int bex = 0;
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
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) {
      sq[k] = fma(a[k], a[k], sq[k]);
      ex[k] = max(ex[k], biased_exp(a[k]));
    }
    if (b != nullptr && lane == 0) bex = max(bex, biased_exp(b[i]));
  }
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    atomicMax(emax + col, ex[2 * k]);
    atomicMax(emax + col + 1, ex[2 * k + 1]);
  }
  if (lane == 0) atomicMax(emax + NC * 64, bex);
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        acc[col] += sq[2 * k];
        acc[col + 1] += sq[2 * k + 1];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npad; i += blockDim.x) {
    const size_t o = (size_t)blockIdx.x * pstride + i;
    colsq_part[o] = (accumulate ? colsq_part[o] : 0.0) + acc[i];
    if (i < n && emax[i] > 0) atomicMax(colexp + i, emax[i]);
  }
  if (threadIdx.x == 0 && emax[NC * 64] > 0) atomicMax(colexp + bslot, emax[NC * 64]);
}

// Fixed-point parameters per column (and b at index npad): with E = the
// largest biased exponent (|a| < 2^(E - 1022)) and L = max(10, bits of the
// longest list), F = (E - 1022) + L - 63, cshift = 1075 + F (the right shift
// of a 53-bit significand with biased exponent e is cshift - e >= 0) and
// cpow = 2^F.  Each term is truncated to a multiple of 2^F, an error below
// 2^F <= 2^(L-62) max |a| (2^-51 max |a| for lists under 2^11 entries), and
// is below 2^(63-L) units in magnitude, so sums of up to 2^L - 1 terms fit in
// 63 bits.  A NaN or Inf (E = 2047) sets st->nonfinite.
__global__ void fixed_params_kernel(const int *__restrict__ colexp, int n, int npad,
                                    const int *__restrict__ lmax, int *cshift, double *cpow,
                                    DevState *st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > npad) return;
  if (j >= n && j < npad) return;
  const int E = max(colexp[j], 1);
  if (colexp[j] == 2047) atomicExch(&st->nonfinite, 1);
  int L = 10;
  while (L < 40 && (1ll << L) <= (long long)*lmax) L++;
  const int F = (E - 1022) + L - 63;
  cshift[j] = 1075 + F;
  cpow[j] = ldexp(1.0, F);
}

// acc += (+-) trunc(|a| / 2^F) with C = 1075 + F, the sign flipped when neg:
// integer operations only.  The shift is PTX shr.b64, which gives 0 for
// shift amounts of 64 or more, so zeros and subnormals (exponent field 0,
// shift 64) and terms below 2^F add 0 with no compare.
__device__ __forceinline__ void add_fixed(long long &acc, double a, int C, unsigned neg) {
  const unsigned hw = (unsigned)__double2hiint(a), lw = (unsigned)__double2loint(a);
  const unsigned e = (hw >> 20) & 0x7ffu;
  const unsigned sh = e ? (unsigned)(C - (int)e) : 64u;
  const unsigned long long mant = ((unsigned long long)((hw & 0xfffffu) | 0x100000u) << 32) | lw;
  unsigned long long t;
  asm("shr.b64 %0, %1, %2;" : "=l"(t) : "l"(mant), "r"(sh));
  const unsigned long long m = 0ull - (unsigned long long)((hw >> 31) ^ neg);  // 0 or ~0
  acc += (long long)((t ^ m) - m);
}

// Fixed-point copy of rows [row0, row1): Q[i ldq + j] = (+-) trunc(|A_ij| /
// 2^F_j) and Qb[i] for b (F from fixed_params_kernel, the terms add_fixed
// forms), so the zeta reads of each entry by the gather are plain 64-bit
// additions.  One warp per row, 64 NC columns per row.
template <int NC, bool VEC>
__global__ void __launch_bounds__(kPassThreads)
    fixed_copy_kernel(const double *__restrict__ A, int64_t lda, int n, const double *__restrict__ b,
                      int npad, const int *__restrict__ cshift, int64_t row0, int64_t row1,
                      long long *__restrict__ Q, int64_t ldq, long long *__restrict__ Qb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int sh[2 * NC];
#pragma unroll
  for (int k = 0; k < NC; k++) {
    const int col = 64 * k + 2 * lane;
    sh[2 * k] = col < n ? cshift[col] : 0;
    sh[2 * k + 1] = col + 1 < n ? cshift[col + 1] : 0;
  }
  const int shb = b != nullptr ? cshift[npad] : 0;
  const int64_t rows = row1 - row0, per = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = row0 + min(rows, (int64_t)blockIdx.x * per), r1 = min(row1, r0 + per);
  for (int64_t i = r0 + warp; i < r1; i += nw) {
    double a[2 * NC];
    load_row<NC, VEC>(A + i * lda, n, lane, a);
    long long q[2 * NC];
#pragma unroll
    for (int k = 0; k < 2 * NC; k++) {
      q[k] = 0;
      add_fixed(q[k], a[k], sh[k], 0u);
    }
    long long *row = Q + i * ldq;
#pragma unroll
    for (int k = 0; k < NC; k++) {
      const int col = 64 * k + 2 * lane;
      if (col + 1 < n) __stcs(reinterpret_cast<longlong2 *>(row + col), make_longlong2(q[2 * k], q[2 * k + 1]));
      else if (col < n) row[col] = q[2 * k];
    }
    if (b != nullptr && lane == 0) {
      long long qb = 0;
      add_fixed(qb, b[i], shb, 0u);
      Qb[i] = qb;
    }
  }
}

// The gather: one warp per (sketch row h, chunk of 64 CH columns) walks h's
// sorted source list and adds or subtracts (the entry's sign, the same for
// the whole warp) the rows' fixed-point values: exact 64-bit integer sums,
// each rounded once to FP64 (times 2^F_j) at the end; accumulate = 1 adds
// them to SAb (rows in chunks).
// RPW sketch rows per warp (only RPW = 1 is launched), each a cursor over
// its list advanced in batches of 32 entries.
template <int CH, int RPW>
__global__ void __launch_bounds__(kGatherWarps * 32, RPW == 2 ? 5 : 1)
    gather_q_kernel(const long long *__restrict__ Q, int64_t ldq, int n,
                    const long long *__restrict__ Qb, int d, int npad,
                    const int64_t *__restrict__ ptr, const uint32_t *__restrict__ src,
                    const double *__restrict__ cpow, double *__restrict__ SAb, int64_t row0,
                    int64_t row1, int accumulate) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.y * CH * 64;
  const int hbase = blockIdx.x * kGatherWarps + warp, hstride = gridDim.x * kGatherWarps;
  const bool dob = (Qb != nullptr && blockIdx.y == 0);
  long long acc[RPW][2 * CH], accb[RPW];
  int64_t p[RPW], pend[RPW];
  bool live[RPW];
#pragma unroll
  for (int r = 0; r < RPW; r++) {
    const int h = hbase + r * hstride;
#pragma unroll
    for (int k = 0; k < 2 * CH; k++) acc[r][k] = 0;
    accb[r] = 0;
    p[r] = pend[r] = 0;
    if (h < d) {
      p[r] = ptr[h];
      pend[r] = ptr[h + 1];
      if (row0 > 0) {
        int64_t lo = p[r], hi = pend[r];
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if ((int64_t)(__ldg(src + mid) & 0x7fffffffu) < row0) lo = mid + 1;
          else hi = mid;
        }
        p[r] = lo;
      }
    }
    live[r] = p[r] < pend[r];
  }
  bool any = true;
  while (any) {
    any = false;
#pragma unroll
    for (int r = 0; r < RPW; r++) {
      if (!live[r]) continue;
      const int64_t p0 = p[r];
      const uint32_t mine = (p0 + lane < pend[r]) ? __ldg(src + p0 + lane) : 0x7fffffffu;
      const unsigned beyond = __ballot_sync(0xffffffffu, (int64_t)(mine & 0x7fffffffu) >= row1);
      const int cnt = beyond ? __ffs(beyond) - 1 : (int)min((int64_t)32, pend[r] - p0);
#pragma unroll 1
      for (int q = 0; q < cnt; q++) {
        const uint32_t e = __shfl_sync(0xffffffffu, mine, q);
        const int64_t i = e & 0x7fffffffu;
        const long long *row = Q + i * ldq + c0;
        long long v[2 * CH];
#pragma unroll
        for (int k = 0; k < CH; k++) {
          const int col = 64 * k + 2 * lane;
          if (c0 + col + 1 < n) {
            const longlong2 t = __ldg(reinterpret_cast<const longlong2 *>(row + col));
            v[2 * k] = t.x;
            v[2 * k + 1] = t.y;
          } else {
            v[2 * k] = (c0 + col < n) ? __ldg(row + col) : 0;
            v[2 * k + 1] = 0;
          }
        }
        const long long vb = (dob && lane == 0) ? __ldg(Qb + i) : 0;
        if (e >> 31) {  // the sign of the entry: the same for the whole warp
#pragma unroll
          for (int k = 0; k < 2 * CH; k++) acc[r][k] -= v[k];
          accb[r] -= vb;
        } else {
#pragma unroll
          for (int k = 0; k < 2 * CH; k++) acc[r][k] += v[k];
          accb[r] += vb;
        }
      }
      p[r] = p0 + 32;
      if (beyond || p[r] >= pend[r]) live[r] = false;
      any = any || live[r];
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; r++) {
    const int h = hbase + r * hstride;
    if (h >= d) continue;
    double *out = SAb + (size_t)h * (n + 1);
#pragma unroll
    for (int k = 0; k < CH; k++) {
      const int col = c0 + 64 * k + 2 * lane;
      if (col < n) out[col] = (accumulate ? out[col] : 0.0) + (double)acc[r][2 * k] * cpow[col];
      if (col + 1 < n)
        out[col + 1] =
            (accumulate ? out[col + 1] : 0.0) + (double)acc[r][2 * k + 1] * cpow[col + 1];
    }
    if (blockIdx.y == 0 && lane == 0)
      out[n] = (accumulate ? out[n] : 0.0) + (dob ? (double)accb[r] * cpow[npad] : 0.0);
  }
}

// ---------------------------------------------------------------------------
// Batched sketch (many problems in one launch, lsq_batch.cu).  CTA g works on
// rows of item cta_item[g]: the scatter form of the pass above, with each
// row's zeta targets drawn inline (each lane of a warp draws the pattern of
// one of 32 consecutive rows, then the warp walks those rows), the hi / lo
// planes written as the rows stream, column sums of squares per CTA.
// zeta <= kBZeta.
// ---------------------------------------------------------------------------
constexpr int kBZeta = 8;

template <int NC>
__device__ void b_sketch_body(const BItem &it, int local, int zeta) {
  __shared__ double acc[4 * 64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = it.n, d = it.d, ldsa = n + 1;
  const int64_t m = it.m;
  const int64_t per = (m + it.ncta - 1) / it.ncta;
  const int64_t r0 = min(m, (int64_t)local * per), r1 = min(m, r0 + per);
  double sq[2 * NC];
#pragma unroll
  for (int k = 0; k < 2 * NC; k++) sq[k] = 0.0;
  for (int64_t i0 = r0 + 32 * warp; i0 < r1; i0 += 32 * nw) {
    int hl[kBZeta];
    uint32_t sbl = 0;
#pragma unroll
    for (int t = 0; t < kBZeta; t++) hl[t] = -1;
    if (i0 + lane < r1) column_pattern<kBZeta>(i0 + lane, d, zeta, it.seed, hl, sbl);
    const int cnt = (int)min((int64_t)32, r1 - i0);
    for (int q = 0; q < cnt; q++) {
      const int64_t i = i0 + q;
      double a[2 * NC];
      load_row<NC, false>(it.A + i * n, n, lane, a);
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        float h0, l0, h1, l1;
        split_rn(a[2 * k], h0, l0);
        split_rn(a[2 * k + 1], h1, l1);
        if (col < n) {
          __stcs(it.Ahi + i * it.ld32 + col, h0);
          __stcs(it.Alo + i * it.ld32 + col, l0);
        }
        if (col + 1 < n) {
          __stcs(it.Ahi + i * it.ld32 + col + 1, h1);
          __stcs(it.Alo + i * it.ld32 + col + 1, l1);
        }
        sq[2 * k] = fma(a[2 * k], a[2 * k], sq[2 * k]);
        sq[2 * k + 1] = fma(a[2 * k + 1], a[2 * k + 1], sq[2 * k + 1]);
      }
      const uint32_t sb = __shfl_sync(0xffffffffu, sbl, q);
      int myh = -1;
#pragma unroll
      for (int t = 0; t < kBZeta; t++) {
        const int ht = __shfl_sync(0xffffffffu, hl[t], q);
        if (lane == t) myh = ht;
      }
      if (lane < zeta && (unsigned)myh < (unsigned)d)
        atomicAdd(it.SAb + (size_t)myh * ldsa + n, flip_sign(it.b[i], (sb >> lane) & 1u));
      for (int t = 0; t < zeta; t++) {
        const int h = __shfl_sync(0xffffffffu, myh, t);
        if ((unsigned)h >= (unsigned)d) continue;
        const bool neg = (sb >> t) & 1u;
        double *dst = it.SAb + (size_t)h * ldsa;
#pragma unroll
        for (int k = 0; k < NC; k++) {
          const int col = 64 * k + 2 * lane;
          if (col < n) atomicAdd(dst + col, flip_sign(a[2 * k], neg));
          if (col + 1 < n) atomicAdd(dst + col + 1, flip_sign(a[2 * k + 1], neg));
        }
      }
    }
  }
  for (int i = threadIdx.x; i < NC * 64; i += blockDim.x) acc[i] = 0.0;
  for (int w = 0; w < nw; w++) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int k = 0; k < NC; k++) {
        const int col = 64 * k + 2 * lane;
        acc[col] += sq[2 * k];
        acc[col + 1] += sq[2 * k + 1];
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < it.npad; i += blockDim.x)
    it.part[(size_t)local * it.npad + i] = acc[i];
}

__global__ void __launch_bounds__(kPassThreads, 2)
    b_sketch_kernel(const BItem *__restrict__ items, const int *__restrict__ cta_item, int zeta) {
  const int idx = cta_item[blockIdx.x];
  const BItem &it = items[idx];
  const int local = blockIdx.x - it.cta0;
  switch (it.npad / 64) {
    case 1: b_sketch_body<1>(it, local, zeta); break;
    case 2: b_sketch_body<2>(it, local, zeta); break;
    case 4: b_sketch_body<4>(it, local, zeta); break;
    default: break;
  }
}

// Column norms of each item from its CTAs' partial sums of squares, and the
// checks of the plan path (non-finite, zero column).
__global__ void b_colnorm_kernel(const BItem *__restrict__ items) {
  const BItem &it = items[blockIdx.x];
  for (int j = threadIdx.x; j < it.n; j += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < it.ncta; g++) s += it.part[(size_t)g * it.npad + j];
    const double nrm = sqrt(s);
    if (!isfinite(nrm)) atomicExch(&it.st->nonfinite, 1);
    if (nrm == 0.0) atomicExch(&it.st->zero_col, 1);
    it.dcol[j] = nrm;
    it.dinv[j] = 1.0 / nrm;
  }
}

// W (d x (n+1), column-major) = the item's sketch scaled (dinv zeta^-1/2 per
// column, zeta^-1/2 for the b column); CTA (x, item) takes the 32 x 32 tiles
// x, x + gridDim.x, ...
__global__ void b_transpose_kernel(const BItem *__restrict__ items, double zinv) {
  __shared__ double tile[32][33];
  const BItem &it = items[blockIdx.y];
  const int ncols = it.n + 1, d = it.d;
  const int tc = (ncols + 31) / 32, th = (d + 31) / 32;
  for (int tt = blockIdx.x; tt < tc * th; tt += gridDim.x) {
    const int c0 = (tt % tc) * 32, h0 = (tt / tc) * 32;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int h = h0 + r, c = c0 + threadIdx.x;
      if (h < d && c < ncols) {
        const double v = it.SAb[(size_t)h * ncols + c];
        if (!isfinite(v)) atomicExch(&it.st->nonfinite, 1);
        tile[r][threadIdx.x] = v;
      }
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
      const int c = c0 + r, h = h0 + threadIdx.x;
      if (h < d && c < ncols) {
        const double sc = (c < it.n) ? it.dinv[c] * zinv : zinv;
        it.W[(size_t)c * d + h] = tile[threadIdx.x][r] * sc;
      }
    }
  }
}

}  // namespace

cudaError_t launch_b_sketch(const BItem *items, const int *cta_item, int grid, int zeta,
                            cudaStream_t s) {
  if (zeta > kBZeta) return cudaErrorInvalidValue;
  b_sketch_kernel<<<grid, kPassThreads, 0, s>>>(items, cta_item, zeta);
  return cudaGetLastError();
}

cudaError_t launch_b_finalize(const BItem *items, int count, int zeta, cudaStream_t s) {
  b_colnorm_kernel<<<count, 256, 0, s>>>(items);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b_transpose_kernel<<<dim3(32, count), dim3(32, 8), 0, s>>>(items, 1.0 / sqrt((double)zeta));
  return cudaGetLastError();
}

int pass_npad(int n) {
  int nc = 1;
  while (nc * 64 < n) nc *= 2;
  return nc * 64;
}

cudaError_t launch_sketch_pattern(int64_t m, int d, int zeta, uint64_t seed, int32_t *rows,
                                  uint32_t *signbits, cudaStream_t s) {
  const int th = 128;
  const int64_t blocks = (m + th - 1) / th;
  pattern_kernel<<<(unsigned)blocks, th, 0, s>>>(m, d, zeta, seed, rows, signbits);
  return cudaGetLastError();
}

template <int NC>
static void sketch_dispatch(bool vec, int grid, cudaStream_t s, const double *A, int64_t lda,
                            int64_t m, int n, const double *b, int d, int zeta,
                            const int32_t *rows, const uint32_t *sb, double *SAb, double *part,
                            int npad, float *Ahi, float *Alo, int64_t ld32) {
  if (vec)
    sketch_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, d, zeta, rows, sb, SAb,
                                                          part, npad, Ahi, Alo, ld32);
  else
    sketch_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, m, n, b, d, zeta, rows, sb,
                                                           SAb, part, npad, Ahi, Alo, ld32);
}

cudaError_t launch_sketch(const double *A, int64_t lda, int64_t m, int n, const double *b, int d,
                          int zeta, const int32_t *rows, const uint32_t *signbits, double *SAb,
                          double *colsq_part, int grid, int npad, float *Ahi, float *Alo,
                          int64_t ld32, cudaStream_t s) {
  const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 2 == 0);
  switch (npad / 64) {
    case 1: sketch_dispatch<1>(vec, grid, s, A, lda, m, n, b, d, zeta, rows, signbits, SAb, colsq_part, npad, Ahi, Alo, ld32); break;
    case 2: sketch_dispatch<2>(vec, grid, s, A, lda, m, n, b, d, zeta, rows, signbits, SAb, colsq_part, npad, Ahi, Alo, ld32); break;
    case 4: sketch_dispatch<4>(vec, grid, s, A, lda, m, n, b, d, zeta, rows, signbits, SAb, colsq_part, npad, Ahi, Alo, ld32); break;
    case 8: sketch_dispatch<8>(vec, grid, s, A, lda, m, n, b, d, zeta, rows, signbits, SAb, colsq_part, npad, Ahi, Alo, ld32); break;
    case 16: sketch_dispatch<16>(vec, grid, s, A, lda, m, n, b, d, zeta, rows, signbits, SAb, colsq_part, npad, Ahi, Alo, ld32); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sketch_finalize(const double *colsq_part, int grid, int npad, int n, int d,
                                   int zeta, int col_scale, const double *SAb, double *W,
                                   double *dcol, double *dinv, DevState *st, cudaStream_t s) {
  colnorm_kernel<<<(n + 255) / 256, 256, 0, s>>>(colsq_part, grid, npad, n, col_scale, dcol, dinv,
                                                 st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 blk(32, 8), grd((n + 1 + 31) / 32, (d + 31) / 32);
  transpose_scale_kernel<<<grd, blk, 0, s>>>(SAb, n, d, dinv, 1.0 / sqrt((double)zeta), W, st);
  return cudaGetLastError();
}


cudaError_t launch_sketch_lists(const int32_t *rows, const uint32_t *signbits, int64_t m, int zeta,
                                int d, int *cnt, int64_t *ptr, uint32_t *src, int *lmax,
                                cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)d, s);
  if (e != cudaSuccess) return e;
  const int64_t mz = m * zeta;
  const unsigned blocks = (unsigned)((mz + 255) / 256);
  tgt_count_kernel<<<blocks, 256, 0, s>>>(rows, mz, d, cnt);
  tgt_scan_kernel<<<1, 1024, 0, s>>>(cnt, d, ptr, lmax);
  tgt_fill_kernel<<<blocks, 256, 0, s>>>(rows, signbits, m, zeta, d, ptr, cnt, src);
  const size_t smem = sizeof(uint32_t) * kSortMax;
  e = ensure_smem_attr((const void *)tgt_sort_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  tgt_sort_kernel<<<d, 512, smem, s>>>(ptr, src);
  return cudaGetLastError();
}

int sketch_list_max() { return kSortMax; }

cudaError_t launch_sketch_prep(const double *A, int64_t lda, int64_t m, int n, const double *b,
                               double *colsq_part, int grid, int npad, int *colexp, float *Ahi,
                               float *Alo, int64_t ld32, cudaStream_t s, int accumulate) {
  cudaError_t e = cudaMemsetAsync(colexp, 0, sizeof(int) * (size_t)(npad + 1), s);
  if (e != cudaSuccess) return e;
  const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 2 == 0);
#define LSQ_PREP(NC, A_, N_, B_, PART_, NP_, EXP_, BSLOT_, HI_, LO_)                              \
  (vec ? prep_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A_, lda, m, N_, B_, PART_, NP_, npad, \
                                                             EXP_, BSLOT_, HI_, LO_, ld32,       \
                                                             accumulate)                         \
       : prep_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A_, lda, m, N_, B_, PART_, NP_,    \
                                                              npad, EXP_, BSLOT_, HI_, LO_,      \
                                                              ld32, accumulate))
  switch (npad / 64) {
    case 1: LSQ_PREP(1, A, n, b, colsq_part, npad, colexp, npad, Ahi, Alo); break;
    case 2: LSQ_PREP(2, A, n, b, colsq_part, npad, colexp, npad, Ahi, Alo); break;
    case 4: LSQ_PREP(4, A, n, b, colsq_part, npad, colexp, npad, Ahi, Alo); break;
    case 8: LSQ_PREP(8, A, n, b, colsq_part, npad, colexp, npad, Ahi, Alo); break;
    case 16: {
      // two passes over column halves: the 1024-column form needs 251 registers
      // (one 8-warp CTA per SM, 3.5 TB/s at 1e6 x 1000); the 512-column form
      // runs two CTAs per SM.  b's exponent goes to colexp[npad] in both.
      LSQ_PREP(8, A, 512, b, colsq_part, 512, colexp, npad, Ahi, Alo);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      LSQ_PREP(8, A + 512, n - 512, nullptr, colsq_part + 512, 512, colexp + 512, npad - 512,
               Ahi ? Ahi + 512 : nullptr, Alo ? Alo + 512 : nullptr);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
#undef LSQ_PREP
  return cudaGetLastError();
}

cudaError_t launch_sketch_gather(const double *A, int64_t lda, int n, const double *b, int d,
                                 int npad, const int64_t *ptr, const uint32_t *src,
                                 const int *colexp, const int *lmax, int *cshift, double *cpow,
                                 double *SAb, DevState *st, cudaStream_t s, int64_t row0,
                                 int64_t row1, int accumulate, long long *Q, long long *Qb,
                                 int64_t ldq, int grid) {
  fixed_params_kernel<<<(npad + 1 + 255) / 256, 256, 0, s>>>(colexp, n, npad, lmax, cshift, cpow,
                                                              st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // 128 columns per warp: a whole column chunk's d warps are resident at
  // once on 152 SMs for d up to ~6000, so they sweep the rows together
  const int ch = npad >= 128 ? 2 : 1;
  const dim3 ggrid((unsigned)((d + kGatherWarps - 1) / kGatherWarps),
                   (unsigned)((n + 64 * ch - 1) / (64 * ch)));
  const int th = kGatherWarps * 32;
  if (Q == nullptr) return cudaErrorInvalidValue;
  {
    const bool vec = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 2 == 0);
#define LSQ_FIXED_COPY(NC)                                                                       \
  (vec ? fixed_copy_kernel<NC, true><<<grid, kPassThreads, 0, s>>>(A, lda, n, b, npad, cshift,   \
                                                                  row0, row1, Q, ldq, Qb)        \
       : fixed_copy_kernel<NC, false><<<grid, kPassThreads, 0, s>>>(A, lda, n, b, npad, cshift,  \
                                                                   row0, row1, Q, ldq, Qb))
    switch (npad / 64) {
      case 1: LSQ_FIXED_COPY(1); break;
      case 2: LSQ_FIXED_COPY(2); break;
      case 4: LSQ_FIXED_COPY(4); break;
      case 8: LSQ_FIXED_COPY(8); break;
      case 16: LSQ_FIXED_COPY(16); break;
      default: return cudaErrorInvalidValue;
    }
#undef LSQ_FIXED_COPY
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // one sketch row per warp: a form with two rows per warp, walked in
    // alternating batches, measured slower at d = 12000 (9.03 against
    // 4.42 ms)
    const long long *qb = b ? Qb : nullptr;
    if (ch == 2)
      gather_q_kernel<2, 1><<<ggrid, th, 0, s>>>(Q, ldq, n, qb, d, npad, ptr, src, cpow, SAb,
                                                 row0, row1, accumulate);
    else
      gather_q_kernel<1, 1><<<ggrid, th, 0, s>>>(Q, ldq, n, qb, d, npad, ptr, src, cpow, SAb,
                                                 row0, row1, accumulate);
    return cudaGetLastError();
  }
}

}  // namespace lsq

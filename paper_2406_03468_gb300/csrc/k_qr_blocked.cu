// Blocked Householder QR of the scaled sketch [SA Sb] (d x ncols,
// column-major, leading dimension d): the factorisation of k_qr.cu's
// column-by-column form (Sec. 2.1; Lemma 6.3's Householder QR), with the
// reflectors of a panel of kQb columns applied to the columns right of it
// at once, in compact-WY form (Schreiber and Van Loan):
//   H_0 H_1 ... H_{b-1} = I - Y T Y^T,  T upper triangular,
//   T_kk = beta_k,  T[0:k, k] = -beta_k T[0:k, 0:k] (Y[:, 0:k]^T y_k),
// so those columns C become C - Y (T^T (Y^T C)).  Reflector k of a panel
// is the unblocked one: for the trailing part x of column k,
//   y_k = x + sign(x_1) ||x|| e_1,  beta_k = 1 / (||x|| (||x|| + |x_1|)),
//   R_kk = -sign(x_1) ||x||,
// and the outputs are those of the column-by-column kernel: R in the upper
// triangle, y_k below the diagonal of column k with its first entry and
// beta_k in vhead[2k], vhead[2k + 1], and Q^T applied to the augmented
// columns (t = Q^T Sb in their first n rows).
//
// GB300 design.  GB300 issues about two FP64 FMAs per clock per SM, so the
// FP64 pipe bounds every part and the work is spread over as many SMs as the
// steps allow.
//  * Panel: one thread-block cluster (16 CTAs where the GPU allows it, else
//    8) holds the panel's trailing rows in shared memory, split into row
//    ranges.  Column k takes one cluster-wide sum: each CTA sends every other
//    CTA its partial [x^T c_j for all panel columns j; row k of the panel]
//    by st.async into the receiver's shared memory, completing a receiver
//    mbarrier that is used once, and adds the partials of all CTAs in rank
//    order (the same bits in every CTA).  x^T c_j gives
//    y_k^T c_j = x^T c_j + sign(x_1) ||x|| c_kj for the columns j > k, and
//    for j < k the Gram entry y_j^T y_k that T's recurrence needs, in the
//    same message.
//  * Trailing update: a cluster per block of 8 columns, one warp per column,
//    its CTAs splitting the rows.  Y^T C is summed across the cluster the
//    same way, multiplied by T^T in shared memory, and each CTA updates its
//    rows (C read from L2 twice, Y through L1).
//  * Lookahead: panel p's reflectors are applied to the next panel's
//    columns first, and the next panel is factored on a second,
//    high-priority stream while the update of panel p's remaining columns
//    runs; two events per panel order the streams.
// Every wait is bounded; on a timeout the kernel records LSQ_ERR_TIMEOUT,
// waits (bounded) for the transfers addressed to its CTA and returns.
#include <atomic>

#include "lsq_cluster.cuh"

namespace lsq {

namespace {

constexpr int kQb = 16;                     // panel width
constexpr int kQbThreads = 256;
constexpr int kQbWarps = kQbThreads / 32;
static_assert(kQb == 2 * kQbWarps, "the panel's warps take two columns each");
constexpr int kMaxClusterQ = 16;
constexpr int kQbMinN = 64;                 // below: the column-by-column kernel
constexpr uint64_t kDrainNs = 2000ull * 1000 * 1000;  // transfers a timed-out CTA still awaits
constexpr size_t kQbSmemMax = 227 * 1024;

__device__ __forceinline__ void note_timeout(DevState *st) {
  atomicCAS(&st->err, 0, (int)LSQ_ERR_TIMEOUT);
}

// The warp totals of 16 per-lane sums by recursive halving: at each of four
// exchanges a lane keeps half of its values and adds its partner's copies of
// them, then one last exchange completes the 32-lane sum.  8 + 4 + 2 + 1 + 1
// FP64 adds per lane instead of 16 x 5 for 16 separate butterflies (each
// FP64 add holds the sub-partition's FP64 pipe about 64 cycles).  Lane L
// returns the total of acc[L >> 1]: bit 4 of L picks the half kept first,
// bits 3, 2 and 1 the next halves.  A fixed order: the same bits every run.
__device__ __forceinline__ double warp_sum16(const double (&acc)[kQb], int lane) {
  static_assert(kQb == 16, "four halvings of 16 values");
  double a8[8], a4[4], a2[2];
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
#pragma unroll
  for (int i = 0; i < 8; i++)
    a8[i] = (h4 ? acc[8 + i] : acc[i]) +
            __shfl_xor_sync(0xffffffffu, h4 ? acc[i] : acc[8 + i], 16);
#pragma unroll
  for (int i = 0; i < 4; i++)
    a4[i] = (h3 ? a8[4 + i] : a8[i]) + __shfl_xor_sync(0xffffffffu, h3 ? a8[i] : a8[4 + i], 8);
#pragma unroll
  for (int i = 0; i < 2; i++)
    a2[i] = (h2 ? a4[2 + i] : a4[i]) + __shfl_xor_sync(0xffffffffu, h2 ? a4[i] : a4[2 + i], 4);
  const double a1 = (h1 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h1 ? a2[0] : a2[1], 2);
  return a1 + __shfl_xor_sync(0xffffffffu, a1, 1);
}

// A double with its sign bit set to `neg`, by its bit pattern (no FP64
// instruction).
__device__ __forceinline__ double with_sign(double x, bool neg) {
  return __hiloint2double((__double2hiint(x) & 0x7fffffff) | (neg ? (int)0x80000000 : 0),
                          __double2loint(x));
}

// The reflector's scalars of a column from the sum of squares sk of its
// trailing part x and its first entry x1: nx = ||x|| = sqrt(sk),
// s = nx with the sign of x1 (+ for x1 = +-0), so that u_1 = x1 + s and
// R_kk = -s, and yy = nx (nx + |x1|) = 1 / beta (beta = 0 when sk = 0).  On
// GB300 every FP64 instruction, a compare included, holds its sub-partition's
// FP64 pipe about 65 cycles and these scalars are on every panel step's
// critical path, so the signs, the absolute value and the zero test are taken
// on the bit patterns.
__device__ __forceinline__ void reflector_scalars(double sk, double x1, double &s, double &yy,
                                                  double &beta) {
  const double nx = sqrt(sk);
  const int xh = __double2hiint(x1);
  const bool neg = xh < 0 && ((xh & 0x7fffffff) | __double2loint(x1)) != 0;
  s = with_sign(nx, neg);
  yy = nx * (nx + with_sign(x1, false));
  const bool zero = ((__double2hiint(sk) & 0x7fffffff) | __double2loint(sk)) == 0;
  beta = zero ? 0.0 : 1.0 / yy;
}

// dynamic shared memory of the panel kernel: 32 doubles for the mbarriers,
// the panel rows (kQb x S), the messages (kQb steps x pc CTAs x 2 kQb), U,
// T, the recursion scratch, the per-step scalars and the partial sums of the
// CTAs' messages
constexpr int kSumWarps = 4;  // warps adding the CTAs' partials of a step
size_t panel_smem_bytes(int S, int pc) {
  return sizeof(double) * (32 + (size_t)kQb * S + (size_t)kQb * pc * 2 * kQb +
                           2 * kQb * kQb + kQb * kQb / 2 + 4 * kQb + kSumWarps * 32);
}

__global__ void __launch_bounds__(kQbThreads, 1)
    qr_panel_kernel(double *__restrict__ W, int d, int kb, int bw, int S,
                    double *__restrict__ vhead, double *__restrict__ Tp, DevState *st,
                    uint64_t timeout_ns) {
  extern __shared__ __align__(16) double psm[];
  const unsigned rank = cluster_rank(), pc = cluster_nranks();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t *bars = reinterpret_cast<uint64_t *>(psm);  // one per panel column
  double *P = psm + 32;                                // column j at P + j S
  double *msg = P + (size_t)kQb * S;                   // step k, CTA r: msg + (k pc + r) 2 kQb
  double *U = msg + (size_t)kQb * pc * 2 * kQb;        // striu(Y^T Y) + diag(1 / beta)
  double *T = U + kQb * kQb;                           // kQb x kQb, column-major (CTA 0)
  double *Xs = T + kQb * kQb;                          // T's recursion scratch (kQb^2 / 2)
  double *wsh = Xs + kQb * kQb / 2;                    // w_j of a step
  double *Tg = wsh + kQb;                              // beta per column
  double *rsh = Tg + kQb;                              // u_1, R_kk of a step
  double *ps = rsh + 2 * kQb;                          // kSumWarps x 32 partial sums
  const int Lp = d - kb;                               // trailing rows of the panel
  const int r0 = (int)rank * S;                        // this CTA's first panel row
  const int nr = max(0, min(S, Lp - r0));
  const int msz = 2 * bw;
  if (tid == 0) {
    for (int k = 0; k < bw; k++) xfer_bar_init(bars + k, 8u * (pc - 1) * (unsigned)msz);
    fence_mbarrier_init_cluster();
  }
  // the panel's rows into shared memory, kBatch loads in flight per thread
  // (one L2 round trip per batch instead of one per element)
  constexpr int kBatch = 4;
  const int tot = bw * nr;
  for (int base = 0; base < tot; base += kBatch * kQbThreads) {
    double v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const int t = base + u * kQbThreads + tid, j = nr > 0 ? t / nr : 0;
      v[u] = t < tot ? W[(size_t)(kb + j) * d + kb + r0 + (t - j * nr)] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const int t = base + u * kQbThreads + tid, j = nr > 0 ? t / nr : 0;
      if (t < tot) P[(size_t)j * S + (t - j * nr)] = v[u];
    }
  }
  for (int i = tid; i < kQb * kQb; i += kQbThreads) U[i] = 0.0;
  __syncthreads();
  cluster_sync_all();  // every barrier is armed before any remote store
  bool ok = true;
  for (int k = 0; k < bw; k++) {
    double *mk = msg + (size_t)k * pc * 2 * kQb;
    double *mine = mk + (size_t)rank * 2 * kQb;
    // rows k.. of the panel; CTA 0 holds rows 0..S-1 (S >= kQb), the others
    // rows beyond them
    const int ilo = rank == 0 ? k : 0;
    const double *x = P + (size_t)k * S;
    {
      // warp w: columns w and w + 8; the two warp sums share their FP64 adds
      // (the first exchange leaves lanes 0-15 with column w's pair sums and
      // lanes 16-31 with column w + 8's, four more halve them to one each)
      const int ja = warp, jb = warp + kQbWarps;
      const double *ca = P + (size_t)ja * S, *cb = P + (size_t)(jb < bw ? jb : ja) * S;
      double a = 0.0, b = 0.0;
      // the step's loops are not unrolled: the FP64 pipe bounds them, and
      // the rolled form measured ~1000 cycles per step faster here
      if (ja < bw) {
#pragma unroll 1
        for (int i = ilo + lane; i < nr; i += 32) a = fma(x[i], ca[i], a);
      }
      if (jb < bw) {
#pragma unroll 1
        for (int i = ilo + lane; i < nr; i += 32) b = fma(x[i], cb[i], b);
      }
      const bool hi = lane >= 16;
      const double send = hi ? a : b, keep = hi ? b : a;
      double v = keep + __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && ja < bw) {
        mine[ja] = v;
        mine[bw + ja] = rank == 0 ? ca[k] : 0.0;
      }
      if (lane == 16 && jb < bw) {
        mine[jb] = v;
        mine[bw + jb] = rank == 0 ? cb[k] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int t = tid; t < (int)(pc - 1) * msz; t += kQbThreads) {
      const unsigned q = (unsigned)(t / msz), e = (unsigned)(t % msz);
      const unsigned dst = q < rank ? q : q + 1;
      st_async_f64(cluster_addr(mine + e, dst), mine[e], cluster_addr(bars + k, dst));
    }
    if (!xfer_wait_limit(bars + k, timeout_ns)) ok = false;
    // the CTAs' messages summed: warp w < kSumWarps adds CTAs
    // w pc / kSumWarps .. in rank order, then warp 0 adds the kSumWarps sums
    // in warp order (a fixed tree: the same bits in every CTA; each FP64 add
    // of a dependent chain costs ~67 cycles, so 4 + 3 adds instead of 16)
    if (warp < kSumWarps && lane < msz) {
      const unsigned per = pc / kSumWarps;
      double s4 = 0.0;
#pragma unroll 1
      for (unsigned r = warp * per; r < (warp + 1) * per; r++) s4 += mk[(size_t)r * 2 * kQb + lane];
      ps[warp * 32 + lane] = s4;
    }
    __syncthreads();
    // warp 0: the reflector, w_j for the columns j > k and the Gram column
    // y_c^T y_k (c < k); the other warps wait at the barrier (GB300 runs FP64
    // sqrt and divide at the FP64 pipe's rate: once per step, not once per
    // warp)
    if (warp == 0) {
      double sv = 0.0;
      if (lane < msz) {
        sv = ps[lane];
        for (int w = 1; w < kSumWarps; w++) sv += ps[w * 32 + lane];
      }
      const double sk = __shfl_sync(0xffffffffu, sv, k);
      const double x1 = __shfl_sync(0xffffffffu, sv, bw + k);
      const double rowj = __shfl_sync(0xffffffffu, sv, (bw + lane) & 31);
      double sn, yy, beta;  // sign(x1) ||x||, y_k^T y_k / 2, beta
      reflector_scalars(sk, x1, sn, yy, beta);
      const double g = fma(sn, rowj, sv);  // y_k^T c_j (j >= k), y_j^T y_k (j < k)
      const double w = beta * g;
      if (lane < bw) {
        if (lane > k) wsh[lane] = w;
        if (lane < k) U[lane + k * kQb] = g;
      }
      if (lane == 0) {
        const double u1 = x1 + sn;
        U[k + k * kQb] = yy;
        Tg[k] = beta;
        rsh[0] = u1;
        rsh[1] = with_sign(sn, __double2hiint(sn) >= 0);  // R_kk = -sn
        if (rank == 0) {
          vhead[2 * (kb + k)] = u1;
          vhead[2 * (kb + k) + 1] = beta;
        }
      }
    }
    __syncthreads();
    // c_j <- c_j - beta y_k (y_k^T c_j) for the panel columns j > k
    const double u1 = rsh[0];
#pragma unroll 1
    for (int j = k + 1 + warp; j < bw; j += kQbWarps) {
      const double wj = wsh[j];
      double *cj = P + (size_t)j * S;
      int i = ilo + lane;
      if (rank == 0 && i == k) {
        cj[k] = fma(-wj, u1, cj[k]);
        i += 32;
      }
#pragma unroll 1
      for (; i < nr; i += 32) cj[i] = fma(-wj, x[i], cj[i]);
    }
    __syncthreads();
    if (tid == 0 && rank == 0) P[(size_t)k * S + k] = rsh[1];
  }
  // T = (striu(Y^T Y) + diag(1 / beta))^{-1} (upper triangular; Schreiber and
  // Van Loan's T, whose recurrence this inverse satisfies), by 2 x 2 block
  // recursion: T_ii = beta_i, then for blocks of size h = 1, 2, 4, 8:
  // T12 = -T11 U12 T22.  No divide; a chain of 2 h FMAs per level.
  if (rank == 0) {
    for (int i = tid; i < kQb * kQb; i += kQbThreads) T[i] = 0.0;
    __syncthreads();
    if (tid < bw) T[tid + tid * kQb] = Tg[tid];
    __syncthreads();
    for (int h = 1; h < kQb; h <<= 1) {
      // blocks at a0 = 2 h q, rows a0..a0+h-1, columns a0+h..a0+2h-1; X = U12 T22
      const int nblk = kQb / (2 * h), per = h * h;
      for (int t = tid; t < nblk * per; t += kQbThreads) {
        const int q = t / per, e = t % per, a = 2 * h * q + e / h, c = 2 * h * q + h + e % h;
        double xv = 0.0;
        for (int l = 2 * h * q + h; l <= c; l++) xv = fma(U[a + l * kQb], T[l + c * kQb], xv);
        Xs[t] = xv;
      }
      __syncthreads();
      for (int t = tid; t < nblk * per; t += kQbThreads) {
        const int q = t / per, e = t % per, a = 2 * h * q + e / h, c = 2 * h * q + h + e % h;
        double v = 0.0;
        for (int l = a; l < 2 * h * q + h; l++) v = fma(T[a + l * kQb], Xs[q * per + (l - 2 * h * q) * h + e % h], v);
        T[a + c * kQb] = -v;
      }
      __syncthreads();
    }
  }
  for (int t = tid; t < tot; t += kQbThreads) {
    const int j = t / nr;
    W[(size_t)(kb + j) * d + kb + r0 + (t - j * nr)] = P[(size_t)j * S + (t - j * nr)];
  }
  if (rank == 0)
    for (int i = tid; i < kQb * kQb; i += kQbThreads) Tp[i] = T[i];
  if (!ok) {
    note_timeout(st);
    for (int k = 0; k < bw; k++) xfer_wait_limit(bars + k, kDrainNs);
  }
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while another may still address it
}

// Columns [c0, c1) of W minus Y (T^T (Y^T C)) for the panel at kb (width
// bw), rows kb..d-1; the cluster's CTAs take rows kb + rank Su .. + Su, a CTA
// CPB columns, kQbWarps / CPB warps per column splitting the CTA's rows.
// Two CTAs per SM at 96 registers leave exactly the registers of one panel CTA
// (64 x 256), so the lookahead panel can start on an SM the update fills.
template <int CPB>
__global__ void __launch_bounds__(kQbThreads, 2)
    qr_update_kernel(double *__restrict__ W, int d, int kb, int bw, int c0, int c1, int Su,
                     const double *__restrict__ vhead, const double *__restrict__ Tp,
                     DevState *st, uint64_t timeout_ns) {
  constexpr int WPC = kQbWarps / CPB, MS = kQb * CPB;
  __shared__ __align__(16) double msg[kMaxClusterQ * MS];
  __shared__ double part[kQbWarps * kQb], wsum[MS], wp[MS], u1s[kQb], Ts[kQb * kQb];
  __shared__ double grp[4 * MS];  // four partial sums per entry (fixed trees below)
  __shared__ uint64_t bar;
  const unsigned rank = cluster_rank(), uc = cluster_nranks();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cw = warp / WPC, sub = warp % WPC;
  const int col = c0 + (int)(blockIdx.x / uc) * CPB + cw;
  const bool has = col < c1;
  const int Lp = d - kb, r0 = (int)rank * Su;
  const int nr = max(0, min(Su, Lp - r0));
  if (tid == 0) {
    xfer_bar_init(&bar, 8u * (uc - 1) * MS);
    fence_mbarrier_init_cluster();
  }
  if (tid < kQb) u1s[tid] = tid < bw ? vhead[2 * (kb + tid)] : 0.0;
  for (int i = tid; i < kQb * kQb; i += kQbThreads) Ts[i] = Tp[i];
  __syncthreads();
  cluster_sync_all();
  const double *Y = W + (size_t)kb * d + kb;  // y_k at Y + k d, rows local to the panel
  double *C = W + (size_t)(has ? col : c0) * d + kb;
  // y_k at panel row gi: stored below the diagonal, u_1 on it, 0 above
  auto yk = [&](int k, int gi) -> double {
    return gi > k ? Y[(size_t)k * d + gi] : (gi == k ? u1s[k] : 0.0);
  };
  double acc[kQb];
#pragma unroll
  for (int k = 0; k < kQb; k++) acc[k] = 0.0;
  if (has) {
    int i = lane + 32 * sub;
    for (; i < nr && r0 + i < bw; i += 32 * WPC) {  // the panel's triangle rows (CTA 0)
      const int gi = r0 + i;
      const double c = C[gi];
#pragma unroll
      for (int k = 0; k < kQb; k++)
        if (k < bw) acc[k] = fma(yk(k, gi), c, acc[k]);
    }
    for (; i < nr; i += 32 * WPC) {
      const int gi = r0 + i;
      const double c = C[gi];
#pragma unroll
      for (int k = 0; k < kQb; k++)
        if (k < bw) acc[k] = fma(__ldg(Y + (size_t)k * d + gi), c, acc[k]);
    }
  }
  {
    const double v = warp_sum16(acc, lane);
    if ((lane & 1) == 0) part[warp * kQb + (lane >> 1)] = v;
  }
  __syncthreads();
  double *mine = msg + (size_t)rank * MS;
  if (tid < MS) {  // this CTA's (Y^T C)[k][c]: the column's warps in order
    const int k = tid / CPB, c = tid % CPB;
    double v = 0.0;
    for (int w = 0; w < WPC; w++) v += part[(c * WPC + w) * kQb + k];
    mine[tid] = v;
  }
  __syncthreads();
  for (int t = tid; t < (int)(uc - 1) * MS; t += kQbThreads) {
    const unsigned q = (unsigned)(t / MS), e = (unsigned)(t % MS);
    const unsigned dst = q < rank ? q : q + 1;
    st_async_f64(cluster_addr(mine + e, dst), mine[e], cluster_addr(&bar, dst));
  }
  const bool ok = xfer_wait_limit(&bar, timeout_ns);
  // the CTAs' partials summed in four groups of ranks, then the four group
  // sums (chains of uc / 4 + 2 dependent adds instead of uc)
  static_assert(4 * MS <= kQbThreads, "a thread per group and entry");
  const int gq = tid / MS, ge = tid % MS;
  if (tid < 4 * MS) {
    const int per = ((int)uc + 3) / 4, rlo = gq * per, rhi = min((int)uc, rlo + per);
    double v = 0.0;
    for (int r = rlo; r < rhi; r++) v += msg[(size_t)r * MS + ge];
    grp[tid] = v;
  }
  __syncthreads();
  if (tid < MS) wsum[tid] = (grp[tid] + grp[MS + tid]) + (grp[2 * MS + tid] + grp[3 * MS + tid]);
  __syncthreads();
  // (T^T (Y^T C))[k][c] = sum_{a <= k} T[a][k] (Y^T C)[a][c], the terms
  // a = 4 q .. 4 q + 3 by group q, then the four group sums
  if (tid < 4 * MS) {
    const int k = ge / CPB, c = ge % CPB, ahi = min(k, 4 * gq + 3);
    double v = 0.0;
    for (int a = 4 * gq; a <= ahi; a++) v = fma(Ts[a + k * kQb], wsum[a * CPB + c], v);
    grp[tid] = v;
  }
  __syncthreads();
  if (tid < MS) wp[tid] = (grp[tid] + grp[MS + tid]) + (grp[2 * MS + tid] + grp[3 * MS + tid]);
  __syncthreads();
  if (has) {
    double wv[kQb];
#pragma unroll
    for (int k = 0; k < kQb; k++) wv[k] = wp[k * CPB + cw];
    int i = lane + 32 * sub;
    for (; i < nr && r0 + i < bw; i += 32 * WPC) {
      const int gi = r0 + i;
      double c = C[gi];
#pragma unroll
      for (int k = 0; k < kQb; k++)
        if (k < bw) c = fma(-yk(k, gi), wv[k], c);
      C[gi] = c;
    }
    for (; i < nr; i += 32 * WPC) {
      const int gi = r0 + i;
      double c = C[gi];
#pragma unroll
      for (int k = 0; k < kQb; k++)
        if (k < bw) c = fma(-__ldg(Y + (size_t)k * d + gi), wv[k], c);
      C[gi] = c;
    }
  }
  if (!ok) {
    note_timeout(st);
    xfer_wait_limit(&bar, kDrainNs);
  }
  __syncthreads();
  cluster_sync_all();
}

std::atomic<int> g_qb_pc[64];  // CTAs of the panel cluster per device (0: not chosen yet)

// The panel cluster: 16 CTAs if a cluster of that size with the panel's
// shared memory can be resident, else 8.
int panel_cluster(int dev, size_t smem16) {
  if (dev < 0 || dev >= 64) return 8;
  if (const int c = g_qb_pc[dev].load()) return c;
  int pc = 8;
  const void *fn = (const void *)qr_panel_kernel;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQbSmemMax) ==
          cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kQbThreads);
    cfg.dynamicSmemBytes = smem16;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters >= 1)
      pc = 16;
  }
  cudaGetLastError();  // a refused query leaves no error behind
  g_qb_pc[dev].store(pc);
  return pc;
}

int rows_per_cta(int Lp, int c) {
  const int s = (Lp + c - 1) / c;
  return s > kQb ? s : kQb;
}

cudaError_t launch_panel(double *W, int d, int kb, int bw, int pc, double *vhead, double *Tp,
                         DevState *st, uint64_t timeout_ns, cudaStream_t s) {
  const int S = rows_per_cta(d - kb, pc);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = pc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(pc);
  cfg.blockDim = dim3(kQbThreads);
  cfg.dynamicSmemBytes = panel_smem_bytes(S, pc);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_panel_kernel, W, d, kb, bw, S, vhead, Tp, st, timeout_ns);
}

template <int CPB>
cudaError_t launch_update(double *W, int d, int kb, int bw, int c0, int c1, int uc,
                          const double *vhead, const double *Tp, DevState *st,
                          uint64_t timeout_ns, cudaStream_t s) {
  if (c1 <= c0) return cudaSuccess;
  const int blocks = (c1 - c0 + CPB - 1) / CPB;
  const int Su = rows_per_cta(d - kb, uc);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = uc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(blocks * uc);
  cfg.blockDim = dim3(kQbThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_update_kernel<CPB>, W, d, kb, bw, c0, c1, Su, vhead, Tp, st,
                            timeout_ns);
}

}  // namespace

bool qr_blocked_ok(int d, int n) {
  if (n < kQbMinN || d < n) return false;
  // the panel's rows must fit the shared memory of the panel cluster
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  const int pc = panel_cluster(dev, panel_smem_bytes(rows_per_cta(d, 16), 16));
  return panel_smem_bytes(rows_per_cta(d, pc), pc) <= kQbSmemMax ||
         panel_smem_bytes(rows_per_cta(d, 8), 8) <= kQbSmemMax;
}

size_t qr_blocked_tws(int n) { return (size_t)((n + kQb - 1) / kQb) * kQb * kQb; }

cudaError_t launch_qr_blocked(double *W, int d, int n, int ncols, double *vhead, double *tws,
                              DevState *st, uint64_t timeout_ns, cudaStream_t s, cudaStream_t sp,
                              cudaEvent_t *ev) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int pc = panel_cluster(dev, panel_smem_bytes(rows_per_cta(d, 16), 16));
  if (panel_smem_bytes(rows_per_cta(d, pc), pc) > kQbSmemMax) pc = 8;
  if (pc == 8) {
    e = cudaFuncSetAttribute((const void *)qr_panel_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQbSmemMax);
    if (e != cudaSuccess) return e;
  }
  // update clusters: the remaining columns 8 per CTA in clusters of 8 CTAs
  // (portable: they pack the GPCs better than 16); the next panel's columns,
  // on the critical path, 2 per CTA in clusters of pc CTAs
  const int uc = 8;
  e = cudaFuncSetAttribute((const void *)qr_update_kernel<4>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)qr_update_kernel<2>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  const int np = (n + kQb - 1) / kQb;
  // ev[0]: the panel stream starts after the work already on s; ev[1..2]:
  // panel p factored (p & 1); ev[3..4]: panel p's remaining columns updated
  if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(sp, ev[0], 0)) != cudaSuccess) return e;
  if ((e = launch_panel(W, d, 0, n < kQb ? n : kQb, pc, vhead, tws, st, timeout_ns, sp)) !=
      cudaSuccess)
    return e;
  if ((e = cudaEventRecord(ev[1], sp)) != cudaSuccess) return e;
  for (int p = 0; p < np; p++) {
    const int kb = p * kQb, bw = n - kb < kQb ? n - kb : kQb;
    const int kn = kb + bw, bwn = kn < n ? (n - kn < kQb ? n - kn : kQb) : 0;
    const double *Tp = tws + (size_t)p * kQb * kQb;
    if (bwn > 0) {
      // the next panel's columns, then the next panel, on the panel stream
      if (p >= 1 && (e = cudaStreamWaitEvent(sp, ev[3 + ((p - 1) & 1)], 0)) != cudaSuccess)
        return e;
      if ((e = launch_update<2>(W, d, kb, bw, kn, kn + bwn, pc, vhead, Tp, st, timeout_ns, sp)) !=
          cudaSuccess)
        return e;
      if ((e = launch_panel(W, d, kn, bwn, pc, vhead, tws + (size_t)(p + 1) * kQb * kQb, st,
                            timeout_ns, sp)) != cudaSuccess)
        return e;
      if ((e = cudaEventRecord(ev[1 + ((p + 1) & 1)], sp)) != cudaSuccess) return e;
    }
    // the remaining columns on s, once panel p is factored
    if ((e = cudaStreamWaitEvent(s, ev[1 + (p & 1)], 0)) != cudaSuccess) return e;
    if ((e = launch_update<4>(W, d, kb, bw, kn + bwn, ncols, uc, vhead, Tp, st, timeout_ns,
                                     s)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(ev[3 + (p & 1)], s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace lsq

// Householder QR of the scaled sketch [SA Sb] (d x (n+1), column-major,
// leading dimension d), giving R (the preconditioner, Sec. 2.1) in the upper
// triangle and t = (Q^T Sb)[0:n] in the last column (the augmented column of
// Alg. 1's sketch-and-solve start).  The paper's analysis assumes Householder
// QR (Lemma 6.3), so this is plain column-by-column Householder: for the
// trailing part x of column k,
//   u = x + sign(x_1) ||x|| e_1,  beta = 2 / ||u||^2 = 1 / (||x|| (||x|| + |x_1|)),
//   R_kk = -sign(x_1) ||x||,  and every later column c <- c - beta u (u^T c),
// with ||u||^2 = 2 ||x|| (||x|| + |x_1|) from the identity, so no FP64
// divide runs per entry.  Reflector k is published in place: rows k+1..d-1
// of column k of W hold u (they are below R's triangle), and u_1, beta go to
// a 2-per-column side array.
//
// GB300 design: one persistent cooperative launch, one CTA per SM.  Each
// column belongs to one CTA for the whole factorisation (snake order, see
// qr_owner) and, when the CTA's columns fit (d = 12n up to n ~ 600), lives
// in that CTA's shared memory from start to end.  There is no grid-wide barrier: the owner of column k
// publishes reflector k with a release store of a per-column flag, and a
// CTA waits (bounded) only for a reflector it has nothing else to do
// without.  Each CTA serves its lowest unfactored column first and catches
// its other columns up while it would otherwise wait (see qr_kernel), so
// the serial chain per column is one column update, one norm and one flag
// hand-off.
#include "lsq_common.cuh"

namespace lsq {

namespace {

constexpr int kQrThreads = 256;
// CTAs per SM.  Columns in shared memory: one, since with the serial
// chain's step fused (apply_build_regs) a second CTA's catch-up FP64 work on
// the same SM slows the chain more than its barrier overlap gains (6.64 vs
// 6.96 ms at d = 6000, n = 500).  Columns in global memory: two, whose
// overlap hides L2 latency (72 vs 106 ms at d = 12000, n = 1000).
constexpr int kQrSmemCtasPerSm = 1;
constexpr int kQrGlobalCtasPerSm = 2;
constexpr int kQrStepCtasPerSm = 2;  // the one-launch-per-column form
constexpr int kQrBatch = 8;  // columns updated together by one CTA

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Reflector of column `col` at step k (rows k..d-1 of col are the current
// trailing column x).  Returns u_1 and beta to every thread, sets col[k] =
// R_kk, and writes R_kk to W's column k row k, u_1 and beta to vhead[2k..];
// with copy_u, also rows k+1..d-1 of col (= u) to W's column k.  Whole CTA.
__device__ void make_reflector(double *col, int k, int d, double *Wk, double *vhead, bool copy_u,
                               double *red, double &uk, double &beta) {
  const int tid = threadIdx.x, nt = blockDim.x;
  double s = 0.0;
  for (int i = k + tid; i < d; i += nt) s = fma(col[i], col[i], s);
  s = block_sum(s, red);
  const double nx = sqrt(s);
  const double x0 = col[k];
  const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
  uk = x0 + sg * nx;
  beta = (nx > 0.0) ? 1.0 / (nx * (nx + fabs(x0))) : 0.0;
  if (copy_u)
    for (int i = k + 1 + tid; i < d; i += nt) Wk[i] = col[i];
  __syncthreads();  // every thread has read col[k]
  if (tid == 0) {
    col[k] = -sg * nx;
    Wk[k] = -sg * nx;
    vhead[2 * k] = uk;
    vhead[2 * k + 1] = beta;
  }
}

// c <- c - beta u (u^T c) for `cnt` <= kQrBatch columns cols[0..cnt), with u
// = (uk, vsrc[k+1..d-1]); VG: vsrc is another CTA's published column (read
// through L2).  Whole CTA.
template <bool VG>
__device__ void apply_reflector(double *const *cols, int cnt, int k, int d, const double *vsrc,
                                double uk, double beta, double *red, double *wsh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int c = 0; c < cnt; c++) {
    const double *col = cols[c];
    double acc = 0.0;
    for (int i = k + 1 + tid; i < d; i += nt) {
      const double vi = VG ? __ldcg(vsrc + i) : vsrc[i];
      acc = fma(vi, col[i], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) red[warp * kQrBatch + c] = acc;
  }
  __syncthreads();
  if (tid < cnt) {
    double sacc = uk * cols[tid][k];
    for (int w = 0; w < nw; w++) sacc += red[w * kQrBatch + tid];
    wsh[tid] = beta * sacc;
  }
  __syncthreads();
  for (int c = 0; c < cnt; c++) {
    double *col = cols[c];
    const double w = wsh[c];
    for (int i = k + 1 + tid; i < d; i += nt) {
      const double vi = VG ? __ldcg(vsrc + i) : vsrc[i];
      col[i] = fma(-w, vi, col[i]);
    }
  }
  if (tid < cnt) cols[tid][k] = fma(-wsh[tid], uk, cols[tid][k]);
  // no closing barrier: callers separate this update from the next reader of
  // other threads' rows (the scheduling barrier of qr_kernel, or an explicit
  // one); a following update of other columns is ordered by its own barriers
}

// The same update with u held in registers: vr[r] = u_i for i = tid + r nt
// (0 outside k < i < d), loaded once per step for all of the CTA's columns.
// The loops over columns run to cnt at run time: an unrolled loop to
// kQrBatch with `c < cnt` guards would issue the guarded-off FP64 FMAs too,
// and GB300's FP64 pipe is the unit that bounds this kernel.
template <int VR>
__device__ void apply_reflector_regs(double *const *cols, int cnt, int k, int d,
                                     const double (&vr)[VR], double uk, double beta, double *red,
                                     double *wsh) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int c = 0; c < cnt; c++) {
    const double *col = cols[c];
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int r = 0; r < VR; r += 2) {
      const int i0 = tid + r * nt, i1 = i0 + nt;
      if (i0 > k && i0 < d) a0 = fma(vr[r], col[i0], a0);
      if (r + 1 < VR && i1 > k && i1 < d) a1 = fma(vr[r + 1], col[i1], a1);
    }
    const double acc = warp_sum(a0 + a1);
    if (lane == 0) red[warp * kQrBatch + c] = acc;
  }
  __syncthreads();
  if (tid < cnt) {
    double sacc = uk * cols[tid][k];
    for (int w = 0; w < nw; w++) sacc += red[w * kQrBatch + tid];
    wsh[tid] = beta * sacc;
  }
  __syncthreads();
  for (int c = 0; c < cnt; c++) {
    double *col = cols[c];
    const double w = wsh[c];
#pragma unroll
    for (int r = 0; r < VR; r++) {
      const int i = tid + r * nt;
      if (i > k && i < d) col[i] = fma(-w, vr[r], col[i]);
    }
  }
  if (tid < cnt) cols[tid][k] = fma(-wsh[tid], uk, cols[tid][k]);
  // no closing barrier: callers separate this update from the next reader of
  // other threads' rows (the scheduling barrier of qr_kernel, or an explicit
  // one); a following update of other columns is ordered by its own barriers
}

// The step on the serial chain: H_k applied to column k+1 (the CTA's pivot)
// fused with building reflector k+1 from it.  The update pass also sums the
// squares of rows k+1.. of the updated column (the norm the reflector needs)
// and writes rows k+2.. to W's column k+1 (the published u), so the chain
// reads the column twice instead of four times.  Whole CTA; as
// apply_reflector_regs then make_reflector(col, k + 1, ..., copy_u = true).
template <int VR>
__device__ void apply_build_regs(double *col, int k, int d, const double (&vr)[VR], double uk,
                                 double beta, double *red, double *wsh, double *Wk1,
                                 double *vhead) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double a0 = 0.0, a1 = 0.0;
#pragma unroll
  for (int r = 0; r < VR; r += 2) {
    const int i0 = tid + r * nt, i1 = i0 + nt;
    if (i0 > k && i0 < d) a0 = fma(vr[r], col[i0], a0);
    if (r + 1 < VR && i1 > k && i1 < d) a1 = fma(vr[r + 1], col[i1], a1);
  }
  const double acc = warp_sum(a0 + a1);
  if (lane == 0) red[warp * kQrBatch] = acc;
  __syncthreads();
  if (tid == 0) {
    double sacc = uk * col[k];
    for (int w = 0; w < nw; w++) sacc += red[w * kQrBatch];
    wsh[0] = beta * sacc;
  }
  __syncthreads();
  const double w = wsh[0];
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int r = 0; r < VR; r++) {
    const int i = tid + r * nt;
    if (i > k && i < d) {
      const double c = fma(-w, vr[r], col[i]);
      col[i] = c;
      if (r & 1) s1 = fma(c, c, s1);
      else s0 = fma(c, c, s0);
      if (i > k + 1) Wk1[i] = c;
    }
  }
  if (tid == 0) col[k] = fma(-w, uk, col[k]);
  const double s = block_sum(s0 + s1, red);  // its barriers also publish col[k + 1]
  const double nx = sqrt(s);
  const double x0 = col[k + 1];
  const double sg = (x0 >= 0.0) ? 1.0 : -1.0;
  const double u1 = x0 + sg * nx;
  const double b1 = (nx > 0.0) ? 1.0 / (nx * (nx + fabs(x0))) : 0.0;
  __syncthreads();  // every thread has read col[k + 1]
  if (tid == 0) {
    col[k + 1] = -sg * nx;
    Wk1[k + 1] = -sg * nx;
    vhead[2 * (k + 1)] = u1;
    vhead[2 * (k + 1) + 1] = b1;
  }
}

// SMEM: the CTA's columns live in shared memory for the whole factorisation.
// VR > 0 (d <= VR * kQrThreads): each thread holds its VR entries of the
// current reflector in registers, so the L2 latency of reading it is paid
// once per update instead of once per loop trip.
//
// Scheduling inside a CTA (thread 0 decides, the CTA executes):
//   * the pivot is the CTA's lowest column whose reflector is not yet built;
//     when it has received H_0 .. H_{j-1} its reflector is built and
//     published at once;
//   * when the reflector the pivot needs next is out, it is applied to the
//     pivot alone if the pivot is the next column to be factored (the
//     critical chain), else to every column of the CTA waiting for it;
//   * while the pivot waits, the CTA catches up its other columns with the
//     reflectors they lack (all already published);
//   * only with nothing else to do does thread 0 wait (bounded) for a flag.
// So the serial chain per column is one column update, one norm and one
// flag hand-off, and the rest of each CTA's FP64 work fills its waits.
constexpr int kQrMaxLocal = 32;  // columns per CTA (bit mask)

// Column ownership of the cooperative kernel: "snake" order over units of
// kQrUnit consecutive columns.  Unit u = j / kQrUnit lies in round
// r = u / G at offset o = u mod G and belongs to CTA o in even rounds and to
// CTA G-1-o in odd ones.  A column's work grows with j (it receives j
// reflectors), and pairing each early unit with a late one evens the CTAs'
// totals (the cyclic order gives the last CTAs of round 0 both heavy units).
// Consecutive columns of one unit share a CTA, so the serial chain passes
// from one CTA to the next once per unit.  Measured at d = 6000, n = 500:
// units of 2 took 8.1 ms against 6.6 ms for units of 1 -- within a unit the
// second column still lacks the previous unit's last reflector when its own
// chain step comes, and that unfused update costs more than the hand-off it
// saves -- so units are single columns.
constexpr int kQrUnit = 1;
__device__ __forceinline__ int qr_owner(int j, int G) {
  const int u = j / kQrUnit, r = u / G, o = u - r * G;
  return (r & 1) ? G - 1 - o : o;
}
// column of CTA me's local column l (increasing with l)
__device__ __forceinline__ int qr_col(int me, int l, int G) {
  const int r = l / kQrUnit, p = l - r * kQrUnit;
  const int u = r * G + ((r & 1) ? G - 1 - me : me);
  return u * kQrUnit + p;
}
// local index of column j at its owner
__device__ __forceinline__ int qr_local(int j, int G) {
  return (j / kQrUnit / G) * kQrUnit + j % kQrUnit;
}
enum { kQrDone = 0, kQrBuild = 1, kQrApply = 2, kQrFail = 3, kQrApplyBuild = 4 };

// The factorisation by G CTAs (this one is `me`); dsm: the columns'
// shared-memory copy (SMEM).  The cooperative kernel runs it with the whole
// grid; the batched one with each item's group of CTAs.
template <bool SMEM, int VR>
__device__ void qr_body(double *__restrict__ W, int d, int n, int ncols, double *__restrict__ vhead,
                        int *flags, int epoch, DevState *st, uint64_t timeout_ns, int G, int me,
                        double *dsm) {
  __shared__ double red[kQrThreads / 32 * kQrBatch];
  __shared__ double wsh[kQrBatch];
  __shared__ int s_act, s_k;
  __shared__ unsigned s_mask;
  const int tid = threadIdx.x, nt = blockDim.x;
  int nloc = 0;  // local columns j = qr_col(me, l, G), increasing with l
  while (qr_col(me, nloc, G) < ncols) nloc++;
  auto colp = [&](int l) -> double * {
    return SMEM ? dsm + (size_t)l * d : W + (size_t)qr_col(me, l, G) * d;
  };
  if (SMEM) {
    for (int l = 0; l < nloc; l++)
      for (int i = tid; i < d; i += nt) dsm[(size_t)l * d + i] = W[(size_t)qr_col(me, l, G) * d + i];
    __syncthreads();
  }
  // thread 0's bookkeeping: reflectors applied per local column, the pivot
  int applied[kQrMaxLocal];
  int piv = 0;  // local index of the lowest unbuilt reflector column (nloc: none)
  if (tid == 0) {
    for (int l = 0; l < kQrMaxLocal; l++) applied[l] = 0;
    while (piv < nloc && qr_col(me, piv, G) >= n) piv++;
  }
  double *cols[kQrBatch];
  for (;;) {
    if (tid == 0) {
      int act = kQrDone, k = 0;
      unsigned mask = 0;
      auto target = [&](int l) { return min(qr_col(me, l, G), n); };
      for (;;) {
        const int jpiv = qr_col(me, piv, G);
        const bool has_piv = piv < nloc && jpiv < n;
        if (has_piv && applied[piv] == jpiv) {
          act = kQrBuild;
          k = jpiv;
          break;
        }
        // the reflector this CTA needs first, and the columns waiting for it.
        // Columns after the pivot never run ahead of it, so with a pivot
        // every reflector below applied[piv] is already out.
        int kneed = n;
        unsigned mneed = 0;
        if (has_piv) {
          kneed = applied[piv];
          if (jpiv == kneed + 1) {
            mneed = 1u << piv;  // the critical chain: the pivot alone
          } else {
            for (int l = piv; l < nloc; l++)
              if (applied[l] == kneed && applied[l] < target(l)) mneed |= 1u << l;
          }
        } else {
          for (int l = 0; l < nloc; l++)
            if (applied[l] < target(l)) kneed = min(kneed, applied[l]);
          if (kneed >= n) {
            act = kQrDone;
            break;
          }
          for (int l = 0; l < nloc; l++)
            if (applied[l] == kneed && applied[l] < target(l)) mneed |= 1u << l;
        }
        if (qr_owner(kneed, G) == me || ld_acquire(flags + kneed) == epoch) {
          act = kQrApply;
          k = kneed;
          mask = mneed;
          // the critical chain with the pivot in shared memory: update and
          // build in one step (apply_build_regs)
          if (SMEM && VR > 0 && has_piv && mneed == (1u << piv) && jpiv == kneed + 1)
            act = kQrApplyBuild;
          break;
        }
        // while it is not out: catch up columns that lag further behind
        int k2 = kneed;
        for (int l = 0; l < nloc; l++)
          if (l != piv && applied[l] < target(l)) k2 = min(k2, applied[l]);
        if (k2 < kneed) {
          act = kQrApply;
          k = k2;
          for (int l = 0; l < nloc; l++)
            if (l != piv && applied[l] == k2 && applied[l] < target(l)) mask |= 1u << l;
          break;
        }
        // nothing to do until reflector kneed is out: bounded wait
        const uint64_t t0 = global_ns();
        bool ok = true;
        while (ld_acquire(flags + kneed) != epoch) {
          if (*(volatile int *)&st->err != 0 || global_ns() - t0 > timeout_ns) {
            atomicCAS(&st->err, 0, (int)LSQ_ERR_TIMEOUT);
            ok = false;
            break;
          }
        }
        if (!ok) {
          act = kQrFail;
          break;
        }
      }
      if (act == kQrBuild || act == kQrApplyBuild) {
        if (act == kQrApplyBuild) applied[piv]++;
        // this column is done once its reflector is out
        do piv++;
        while (piv < nloc && qr_col(me, piv, G) >= n);
      } else if (act == kQrApply) {
        for (int l = 0; l < nloc; l++)
          if (mask & (1u << l)) applied[l]++;
      }
      s_act = act;
      s_k = k;
      s_mask = mask;
    }
    __syncthreads();
    const int act = s_act, k = s_k;
    const unsigned mask = s_mask;
    if (act == kQrDone || act == kQrFail) break;
    if (act == kQrBuild) {
      double uk, beta;
      make_reflector(colp(qr_local(k, G)), k, d, W + (size_t)k * d, vhead, SMEM, red, uk, beta);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(flags + k, epoch);
      }
      continue;
    }
    if (mask == 0) {  // (not produced by the schedule above; keeps the barrier pattern safe)
      __syncthreads();
      continue;
    }
    // apply H_k to the columns in mask; u from this CTA's own copy or the published one
    const bool own = (qr_owner(k, G) == me);
    if (act == kQrApplyBuild) {
      if (VR > 0) {
        const double uk = __ldcg(vhead + 2 * k), beta = __ldcg(vhead + 2 * k + 1);
        const double *vk = own ? colp(qr_local(k, G)) : W + (size_t)k * d;
        double vr[VR > 0 ? VR : 1];
#pragma unroll
        for (int r = 0; r < (VR > 0 ? VR : 1); r++) {
          const int i = tid + r * nt;
          vr[r] = (i > k && i < d) ? (own ? vk[i] : __ldcg(vk + i)) : 0.0;
        }
        apply_build_regs(colp(qr_local(k + 1, G)), k, d, vr, uk, beta, red, wsh,
                         W + (size_t)(k + 1) * d, vhead);
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(flags + k + 1, epoch);
      }
      continue;
    }
    const double uk = __ldcg(vhead + 2 * k), beta = __ldcg(vhead + 2 * k + 1);
    const double *vk = own ? colp(qr_local(k, G)) : W + (size_t)k * d;
    double vr[VR > 0 ? VR : 1];
    if (VR > 0) {
#pragma unroll
      for (int r = 0; r < (VR > 0 ? VR : 1); r++) {
        const int i = tid + r * nt;
        vr[r] = (i > k && i < d) ? (own ? vk[i] : __ldcg(vk + i)) : 0.0;
      }
    }
    unsigned rest = mask;
    while (rest) {
      int cnt = 0;
      while (rest && cnt < kQrBatch) {
        const int l = __ffs(rest) - 1;
        rest &= rest - 1;
        cols[cnt++] = colp(l);
      }
      if (VR > 0) apply_reflector_regs(cols, cnt, k, d, vr, uk, beta, red, wsh);
      else if (own) apply_reflector<false>(cols, cnt, k, d, vk, uk, beta, red, wsh);
      else apply_reflector<true>(cols, cnt, k, d, vk, uk, beta, red, wsh);
    }
  }
  if (SMEM && s_act == kQrDone) {
    // R rows above the diagonal of the reflector columns, and the augmented
    // columns whole (rows k..d-1 of reflector column k went out at publish).
    for (int l2 = 0; l2 < nloc; l2++) {
      const int j = qr_col(me, l2, G);
      const int iend = (j < n) ? j : d;
      for (int i = tid; i < iend; i += nt) W[(size_t)j * d + i] = dsm[(size_t)l2 * d + i];
    }
  }
}

template <bool SMEM, int VR>
__global__ void __launch_bounds__(kQrThreads, SMEM ? kQrSmemCtasPerSm : kQrGlobalCtasPerSm)
    qr_kernel(double *__restrict__ W, int d, int n, int ncols, double *__restrict__ vhead,
              int *flags, int epoch, DevState *st, uint64_t timeout_ns) {
  extern __shared__ double dsm[];
  qr_body<SMEM, VR>(W, d, n, ncols, vhead, flags, epoch, st, timeout_ns, gridDim.x, blockIdx.x,
                    dsm);
}

// Batched form: one cooperative launch factors every item's sketch, item i on
// its group of CTAs (cta_item map; cta0 / ncta of the item's QR group), with
// the columns in global memory (L2) and the reflector in registers (VR = 12
// covers d = 12 n <= 3072).  Flags per item; waits bounded as above.
__global__ void __launch_bounds__(kQrThreads, kQrGlobalCtasPerSm)
    b_qr_kernel(const BItem *__restrict__ items, const int *__restrict__ qmap, int epoch,
                uint64_t timeout_ns) {
  const int idx = qmap[blockIdx.x];
  if (idx < 0) return;
  const BItem &it = items[idx];
  const int me = blockIdx.x - it.qcta0, G = it.qncta;
  if (it.d <= 8 * kQrThreads)
    qr_body<false, 8>(it.W, it.d, it.n, it.n + 1, it.vhead, it.qflag, epoch, it.st, timeout_ns, G,
                      me, nullptr);
  else
    qr_body<false, 12>(it.W, it.d, it.n, it.n + 1, it.vhead, it.qflag, epoch, it.st, timeout_ns,
                       G, me, nullptr);
}

// Non-cooperative form for concurrent solves (served requests): one launch
// per column step, the kernel boundary standing in for the flags.  Column j
// belongs to CTA j mod G; the owner of column k+1 applies H_k to it and
// publishes reflector k+1 within step k (lookahead); the reflectors are
// published as in the cooperative kernel; columns stay in global memory.
__device__ void qr_step_body(double *__restrict__ W, int d, int n, int ncols,
                             double *__restrict__ vhead, int k, int G, int me) {
  __shared__ double red[kQrThreads / 32 * kQrBatch];
  __shared__ double wsh[kQrBatch];
  const int nloc = (ncols - me + G - 1) / G;
  auto colp = [&](int l) -> double * { return W + (size_t)(me + l * G) * d; };
  double uk, beta;
  if (k < 0) {  // prologue: reflector 0
    if (me == 0) make_reflector(colp(0), 0, d, W, vhead, false, red, uk, beta);
    return;
  }
  uk = __ldcg(vhead + 2 * k);
  beta = __ldcg(vhead + 2 * k + 1);
  const double *vk = W + (size_t)k * d;
  double *cols[kQrBatch];
  const int l0 = (k + 1 > me) ? (k + 1 - me + G - 1) / G : 0;
  int l = l0;
  if (k + 1 < n && (k + 1) % G == me && l < nloc) {
    cols[0] = colp(l);
    apply_reflector<true>(cols, 1, k, d, vk, uk, beta, red, wsh);
    __syncthreads();  // the norm below reads rows other threads just updated
    double u1, b1;
    make_reflector(colp(l), k + 1, d, W + (size_t)(k + 1) * d, vhead, false, red, u1, b1);
    l++;
  }
  while (l < nloc) {
    int cnt = 0;
    for (; cnt < kQrBatch && l < nloc; cnt++, l++) cols[cnt] = colp(l);
    apply_reflector<true>(cols, cnt, k, d, vk, uk, beta, red, wsh);
  }
}

__global__ void __launch_bounds__(kQrThreads)
    qr_step_kernel(double *__restrict__ W, int d, int n, int ncols, double *__restrict__ vhead,
                   int k) {
  qr_step_body(W, d, n, ncols, vhead, k, gridDim.x, blockIdx.x);
}

// The same step for every item of a batch (grid y = item); items with fewer
// columns than the step are done.
__global__ void __launch_bounds__(kQrThreads)
    b_qr_step_kernel(const BItem *__restrict__ items, int k) {
  const BItem &it = items[blockIdx.y];
  if (k >= it.n) return;
  qr_step_body(it.W, it.d, it.n, it.n + 1, it.vhead, k, gridDim.x, blockIdx.x);
}

__global__ void extract_r_kernel(const double *__restrict__ W, int d, int n, int nb, double *Rcm,
                                 double *Rrm, double *rinv, double *t) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)n * n;
  if (idx < nn) {
    const int j = (int)(idx / n), i = (int)(idx % n);  // column j, row i
    const double v = (i <= j) ? W[(size_t)j * d + i] : 0.0;
    Rcm[(size_t)j * n + i] = v;
    Rrm[(size_t)i * n + j] = v;
  }
  if (idx < n) rinv[idx] = 1.0 / W[(size_t)idx * d + idx];
  // t (n x nb, column-major) = rows 0..n-1 of the augmented columns
  if (idx < (int64_t)n * nb) {
    const int c = (int)(idx / n), i = (int)(idx % n);
    t[idx] = W[(size_t)(n + c) * d + i];
  }
}

}  // namespace

int qr_grid(int ncols, int nsm) {
  const int units = (ncols + kQrUnit - 1) / kQrUnit;
  return units < kQrGlobalCtasPerSm * nsm ? units : kQrGlobalCtasPerSm * nsm;
}
int qr_step_grid(int ncols, int nsm) {
  return ncols < kQrStepCtasPerSm * nsm ? ncols : kQrStepCtasPerSm * nsm;
}

// Largest dynamic shared memory the columns may use (227 KB opt-in minus the static part).
constexpr size_t kQrSmemMax = 225 * 1024;

template <bool SMEM, int VR>
cudaError_t launch_qr_t(void **args, int grid, size_t smem, cudaStream_t s) {
  const void *fn = (const void *)qr_kernel<SMEM, VR>;
  if (SMEM) {
    cudaError_t e = ensure_smem_attr(fn, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kQrThreads), args, SMEM ? smem : 0, s);
}

template <bool SMEM>
cudaError_t launch_qr_vr(void **args, int d, int grid, size_t smem, cudaStream_t s) {
  if (d <= 8 * kQrThreads) return launch_qr_t<SMEM, 8>(args, grid, smem, s);
  if (d <= 12 * kQrThreads) return launch_qr_t<SMEM, 12>(args, grid, smem, s);
  if (d <= 16 * kQrThreads) return launch_qr_t<SMEM, 16>(args, grid, smem, s);
  if (d <= 24 * kQrThreads) return launch_qr_t<SMEM, 24>(args, grid, smem, s);
  return launch_qr_t<SMEM, 0>(args, grid, smem, s);
}

cudaError_t launch_qr(double *W, int d, int n, int ncols, double *vhead, int *flags, int epoch,
                      DevState *st, int grid, uint64_t timeout_ns, cudaStream_t s,
                      const QrBlocked *qb) {
  if (qb != nullptr && qr_blocked_ok(d, n))
    return launch_qr_blocked(W, d, n, ncols, vhead, qb->tws, st, timeout_ns, s, qb->sp,
                             const_cast<cudaEvent_t *>(qb->ev));
  void *args[] = {&W, &d, &n, &ncols, &vhead, &flags, &epoch, &st, &timeout_ns};
  // grid: CTAs at kQrGlobalCtasPerSm per SM (qr_grid).  Columns in shared
  // memory at kQrSmemCtasPerSm CTAs per SM if they fit, else in global
  // memory (L2) at kQrGlobalCtasPerSm per SM.
  // local columns per CTA: whole units, dealt over the g CTAs
  auto nloc_for = [&](int g) {
    const int units = (ncols + kQrUnit - 1) / kQrUnit;
    return ((units + g - 1) / g) * kQrUnit;
  };
  auto smem_for = [&](int g) { return (size_t)nloc_for(g) * d * sizeof(double); };
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int units = (ncols + kQrUnit - 1) / kQrUnit;
  const int g1 = units < kQrSmemCtasPerSm * nsm ? units : kQrSmemCtasPerSm * nsm;
  if (kQrSmemCtasPerSm * smem_for(g1) <= kQrSmemMax && nloc_for(g1) <= kQrMaxLocal) {
    void *args1[] = {&W, &d, &n, &ncols, &vhead, &flags, &epoch, &st, &timeout_ns};
    return launch_qr_vr<true>(args1, d, g1, smem_for(g1), s);
  }
  if (nloc_for(grid) > kQrMaxLocal) return cudaErrorInvalidConfiguration;
  return launch_qr_vr<false>(args, d, grid, 0, s);
}

cudaError_t launch_qr_stepwise(double *W, int d, int n, int ncols, double *vhead, int grid,
                               cudaStream_t s) {
  for (int k = -1; k < n; k++) {
    qr_step_kernel<<<grid, kQrThreads, 0, s>>>(W, d, n, ncols, vhead, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_b_qr(const BItem *items, const int *qmap, int grid, int epoch,
                        uint64_t timeout_ns, cudaStream_t s) {
  void *args[] = {(void *)&items, (void *)&qmap, &epoch, &timeout_ns};
  return cudaLaunchCooperativeKernel((const void *)b_qr_kernel, dim3(grid), dim3(kQrThreads), args,
                                     0, s);
}

int b_qr_max_ctas(int nsm) { return kQrGlobalCtasPerSm * nsm; }
int b_qr_min_ctas(int n) { return (n + 1 + kQrMaxLocal - 1) / kQrMaxLocal; }

cudaError_t launch_b_qr_step(const BItem *items, int count, int qcta, int k, cudaStream_t s) {
  b_qr_step_kernel<<<dim3(qcta, count), kQrThreads, 0, s>>>(items, k);
  return cudaGetLastError();
}

cudaError_t launch_extract_r(const double *W, int d, int n, int nb, double *Rcm, double *Rrm,
                             double *rinv, double *t, cudaStream_t s) {
  const int64_t nn = (int64_t)n * (n > nb ? n : nb);
  const int th = 256;
  extract_r_kernel<<<(unsigned)((nn + th - 1) / th), th, 0, s>>>(W, d, n, nb, Rcm, Rrm, rinv, t);
  return cudaGetLastError();
}

}  // namespace lsq

// Device helpers shared by the streaming passes over the FP32 planes of A
// (k_pass.cu, k_multi_df.cu): error-free FP32 arithmetic (TwoSum, exact
// widening to FP64, packed f32x2 double-float steps), mbarrier operations
// and TMA bulk copies.  Internal to liblsq; nothing here is part of the ABI.
#pragma once

#include <stdint.h>

#include "lsq_common.cuh"

namespace lsq {

// Knuth's TwoSum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Exact FP32 -> FP64 widening with integer operations (normal and zero inputs).
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0) return 0.0;
  const unsigned hw = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
  return __hiloint2double((int)hw, (int)(b << 29));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"((unsigned)__cvta_generic_to_shared(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase, uint64_t limit_ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, phase))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

// L2 policy for data read once (the planes of A stream through L2 dozens of
// times per solve and would otherwise evict R and the partial sums the small
// kernels between passes read).
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                         uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
      "l"(src), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(bar)), "l"(pol)
      : "memory");
}

// Packed FP32 pairs (two columns per 64-bit register, the lower one in the
// low word): sm_100-class add / sub / mul / fma .rn.f32x2 round each half as
// the scalar instruction would, at one issue slot per two elements.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
  f2_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
  f2_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  return ((f2_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float f2_lo(f2_t v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(f2_t v) { return __uint_as_float((unsigned)(v >> 32)); }
// One double-float accumulation step on a pair: (s, l) += (a * b exactly,
// with the cross terms a * bl + al * b), given bn = -b.  The product's
// rounding error comes from fma(a, b, -p) with -p = a * bn; the TwoSum adds p
// as s - (-p).  Every operation is the scalar algorithm's, per half.
__device__ __forceinline__ void f2_dd_step(f2_t &s, f2_t &l, f2_t a, f2_t al, f2_t b, f2_t bl,
                                           f2_t bn) {
  const f2_t pn = f2_mul(a, bn);
  const f2_t c = f2_fma(a, bl, f2_fma(al, b, f2_fma(a, b, pn)));
  const f2_t s1 = f2_sub(s, pn);
  const f2_t bb = f2_sub(s1, s);
  const f2_t er = f2_sub(f2_sub(s, f2_sub(s1, bb)), f2_add(pn, bb));
  s = s1;
  l = f2_add(l, f2_add(er, c));
}

// Renormalisation of a packed double-float pair by TwoSum (exact whatever
// the magnitudes): (s, l) <- (fl(s + l), the exact remainder).
__device__ __forceinline__ void f2_renorm(f2_t &s, f2_t &l) {
  const f2_t t = f2_add(s, l);
  const f2_t bb = f2_sub(t, s);
  l = f2_add(f2_sub(s, f2_sub(t, bb)), f2_sub(l, bb));
  s = t;
}

}  // namespace lsq

// vfe_tc_common.cuh -- device helpers shared by the tensor-core kernels
// (mbarrier waits, TMA, tcgen05 MMA and TMEM access, the exact integer
// arithmetic of the epilogues).  Included by the .cu files of the TC path.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "vfe_internal.h"

namespace vfe_tc {

constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits give up after ~2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of a completed phase (acquire when it succeeds).
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 256; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_u(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                           int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(0)
      : "memory");
}

__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// Issued by every lane of a converged warp; one elected lane executes the
// instruction, so descriptors formed as a base plus constants can stay in
// uniform registers (the issue then keeps pace with the tensor pipe).
__device__ __forceinline__ void mma_f16_elect(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit_elect(uint64_t *bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t &a, uint32_t &b, uint32_t &c,
                                         uint32_t &d) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// Load 12 consecutive columns (x8 at c, x4 at c + 8 when c = 0 mod 8, else x4
// at c and x8 at c + 4) of this warp's lanes.
__device__ __forceinline__ void tmem_ld12(uint32_t taddr, bool first8, uint32_t *r) {
  if (first8) {
    tmem_ld8(taddr, r);
    tmem_ld4(taddr + 8, r[8], r[9], r[10], r[11]);
  } else {
    tmem_ld4(taddr, r[0], r[1], r[2], r[3]);
    tmem_ld8(taddr + 4, r + 4);
  }
}

// Wait for this thread's TMEM loads; the loaded registers pass through the
// statement so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait_ld12(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11])
               :
               : "memory");
}

// Wait for this thread's TMEM loads, passing 8 loaded registers through.
__device__ __forceinline__ void tmem_wait_ld8(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

// Wait for this thread's TMEM loads, passing 4 loaded registers through.
__device__ __forceinline__ void tmem_wait_ld4(uint32_t *r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3])
               :
               : "memory");
}

// Store the value v into 4 consecutive columns of this warp's lanes.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %1, %1, %1};" ::"r"(taddr), "r"(v)
               : "memory");
}

// Store the value v into 8 consecutive columns of this warp's lanes.
__device__ __forceinline__ void tmem_st8v(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
                   taddr),
               "r"(v)
               : "memory");
}

// Store 8 consecutive columns of this warp's lanes, and wait for the stores.
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
                   taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
               "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// round(v / 2^s), halves toward +inf, for |v| < 2^62; v * 2^-s for s <= 0
__device__ __forceinline__ int64_t shr_round(int64_t v, int s) {
  if (s <= 0) return (int64_t)((uint64_t)v << min(-s, 63));
  if (s >= 63) return 0;
  return (v + ((int64_t)1 << (s - 1))) >> s;
}

// exact small integer -> fp32 (|d| < 2^22) without a conversion instruction
__device__ __forceinline__ float int_to_f32_exact(int d) {
  return __int_as_float(TC_MAGIC_BITS + d) - 12582912.0f;
}

// ---------------------------------------------------------------------------
// Epilogue arithmetic.
// ---------------------------------------------------------------------------
// One stage of the exact recombination P = sum_s 2^(11 s) D_s of the
// magic-biased accumulator words w_s = 0x4B400000 + D_s, Horner order over the
// stages; the biases of all five words are removed at the end by
// recomb_finish (mod 2^64 arithmetic is exact because P fits in int64).
template <int S>
__device__ __forceinline__ void recomb_stage(uint64_t &t, uint32_t w) {
  if constexpr (S == 0) {
    t = (uint64_t)w;
  } else if constexpr (S == 1) {
    asm("mad.wide.u32 %0, %1, 2048, %0;" : "+l"(t) : "r"(w));
  } else if constexpr (S == 2) {
    asm("mad.wide.u32 %0, %1, 4194304, %0;" : "+l"(t) : "r"(w));
  } else if constexpr (S == 3) {
    t += (uint64_t)(w << 1) << 32;
  } else {
    t += (uint64_t)(w << 12) << 32;
  }
}
__device__ __forceinline__ int64_t recomb_finish(uint64_t t) {
  constexpr uint64_t kBias = (uint64_t)TC_MAGIC_BITS *
                             (1ull + 2048ull + 4194304ull + 8589934592ull + 17592186044416ull);
  return (int64_t)(t - kBias);
}

// floor((P A + Q B) / 2^63) within 4 units, for any int64 P, Q and the
// material multipliers A = A1 2^31 + A0, B = B1 2^31 + B0 (0 <= A0, B0 < 2^31;
// 0 <= A1, B1 < 2^30).  With P = p1 2^32 + p0 (p1 signed, p0 unsigned):
//   P A / 2^63 = p1 A1 + p1 A0 / 2^31 + p0 A1 / 2^32 + p0 A0 / 2^63,
// and likewise for Q B.  The three leading terms of both products are summed
// as p1 A1 + q1 B1, floor((p1 A0 + q1 B0) / 2^31) (|.| < 2^63) and the high
// word of p0 A1 + q0 B1 (< 2^63); the last terms (< 2 together) are dropped.
__device__ __forceinline__ int64_t mul2_hi63(int64_t P, int64_t Q, int A1, int A0, int B1,
                                             int B0) {
  int64_t r;
  asm("{\n"
      " .reg .u32 p0, p1, q0, q1, l0, l1;\n"
      " .reg .u64 lo, t3;\n"
      " .reg .s64 mid, res;\n"
      " mov.b64 {p0, p1}, %1;\n"
      " mov.b64 {q0, q1}, %2;\n"
      " mul.wide.u32 lo, p0, %3;\n"
      " mad.wide.u32 lo, q0, %5, lo;\n"
      " mov.b64 {l0, l1}, lo;\n"
      " cvt.u64.u32 t3, l1;\n"
      " mul.wide.s32 mid, p1, %4;\n"
      " mad.wide.s32 mid, q1, %6, mid;\n"
      " shr.s64 mid, mid, 31;\n"
      " mul.wide.s32 res, p1, %3;\n"
      " mad.wide.s32 res, q1, %5, res;\n"
      " add.s64 res, res, mid;\n"
      " add.s64 %0, res, t3;\n"
      "}\n"
      : "=l"(r)
      : "l"(P), "l"(Q), "r"(A1), "r"(A0), "r"(B1), "r"(B0));
  return r;
}

// floor(P C / 2^63) within 2 units for 0 <= C = C1 2^31 + C0 < 2^62 and
// |P| < 2^63: the same limb products as mul2_hi63 for one term.
__device__ __forceinline__ int64_t mul_hi63(int64_t P, int C1, int C0) {
  int64_t r;
  asm("{\n"
      " .reg .u32 p0, p1;\n"
      " .reg .u64 lo, res;\n"
      " .reg .s64 mid;\n"
      " mov.b64 {p0, p1}, %1;\n"
      " mul.wide.u32 lo, p0, %2;\n"
      " shr.u64 lo, lo, 1;\n"
      " mul.wide.s32 mid, p1, %3;\n"
      " add.s64 mid, mid, lo;\n"
      " shr.s64 mid, mid, 31;\n"
      " mul.wide.s32 res, p1, %2;\n"
      " add.s64 %0, res, mid;\n"
      "}\n"
      : "=l"(r)
      : "l"(P), "r"(C1), "r"(C0));
  return r;
}

// round(S C / 2^R) for 1 <= R <= 63, S signed, 0 <= C < 2^63, from the exact
// 128-bit product: add 2^(R-1), then the 64 bits starting at bit R
__device__ __forceinline__ int64_t mul_shr_round(int64_t S, int64_t C, int R) {
  int64_t r;
  asm("{\n"
      " .reg .u64 lo, hi, one, rnd;\n"
      " .reg .u32 sl, sr;\n"
      " mul.lo.u64 lo, %1, %2;\n"
      " mul.hi.s64 hi, %1, %2;\n"
      " sub.u32 sl, %3, 1;\n"
      " shl.b64 rnd, 1, sl;\n"
      " add.cc.u64 lo, lo, rnd;\n"
      " addc.u64 hi, hi, 0;\n"
      " shr.b64 lo, lo, %3;\n"
      " sub.u32 sr, 64, %3;\n"
      " shl.b64 hi, hi, sr;\n"
      " or.b64 %0, lo, hi;\n"
      "}\n"
      : "=l"(r)
      : "l"(S), "l"(C), "r"(R));
  return r;
}

}  // namespace vfe_tc

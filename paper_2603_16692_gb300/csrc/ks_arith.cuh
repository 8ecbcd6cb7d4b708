// 64-bit modular arithmetic for the KeySwitch kernels (device side).
//
// Moduli are < 2^62. Three reductions are used:
//  * Shoup multiplication by a constant w with w' = floor(w 2^64 / m):
//      y*w - umulhi(y, w')*m  lies in [0, 2m) for any y < 2^64.
//  * Montgomery reduction (REDC) of a 128-bit sum T < m 2^64:
//      (T + u m) / 2^64 with u = T_lo * (-m^-1) mod 2^64, result in [0, 2m).
//    Basis-conversion and key-multiply sums are accumulated exactly in 128 bits
//    and reduced once; constants carry the 2^64 factors that REDC removes.
//  * Lazy ranges: forward butterflies keep values in [0, 4m), inverse ones in
//    [0, 2m) (Harvey's butterflies); outputs are made canonical at the end.
#pragma once
#include <cstdint>

typedef unsigned long long u64;

struct U128 {
  u64 lo, hi;
};

__device__ __forceinline__ void mac128(U128 &acc, u64 a, u64 b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
      "madc.hi.u64 %1, %2, %3, %1;"
      : "+l"(acc.lo), "+l"(acc.hi)
      : "l"(a), "l"(b));
}

// T * 2^-64 mod m in [0, 2m) for T < m * 2^64; minv = -m^-1 mod 2^64.
__device__ __forceinline__ u64 redc(const U128 &t, u64 m, u64 minv) {
  const u64 u = t.lo * minv;
  return t.hi + __umul64hi(u, m) + (t.lo != 0ull ? 1ull : 0ull);
}

// y * w mod m in [0, 2m).
__device__ __forceinline__ u64 shoup(u64 y, u64 w, u64 wp, u64 m) {
  const u64 q = __umul64hi(y, wp);
  return y * w - q * m;
}

__device__ __forceinline__ u64 csub(u64 x, u64 m) { return x >= m ? x - m : x; }

// High 64 bits of y*wp, under-estimated by at most 2: yh*wh plus the high words of
// the two cross products; the low x low product and the carry out of the low words
// of the cross products are dropped (each worth at most 1).
__device__ __forceinline__ u64 mulhi_approx(u64 y, u64 wp) {
  const uint32_t yl = (uint32_t)y, yh = (uint32_t)(y >> 32);
  const uint32_t wl = (uint32_t)wp, wh = (uint32_t)(wp >> 32);
  u64 t1, t2, h;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(t1) : "r"(yl), "r"(wh));
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(t2) : "r"(yh), "r"(wl));
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(h) : "r"(yh), "r"(wh), "l"((t1 >> 32) + (t2 >> 32)));
  return h;
}

// y * w mod m in [0, 4m) with the approximate quotient (Shoup's bound 2m plus 2m).
__device__ __forceinline__ u64 shoup4(u64 y, u64 w, u64 wp, u64 m) {
  return y * w - mulhi_approx(y, wp) * m;
}

// x mod m for any x < 2^64 (Barrett with mu = floor(2^64 / m)), canonical.
__device__ __forceinline__ u64 reduce_full(u64 x, u64 m, u64 mu) {
  const u64 r = x - __umul64hi(x, mu) * m;  // in [0, 2m)
  return r >= m ? r - m : r;
}

// Bulk prefetch of `bytes` (multiple of 16, 16-byte aligned) from global memory into
// L2 by the TMA unit; no registers or shared memory are involved.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 eviction priorities (createpolicy): twiddle tables are read by every launch and
// should stay in L2 (evict_last); key words are read once per KeySwitch (evict_first).
__device__ __forceinline__ u64 l2_keep() {
  u64 p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ u64 l2_stream() {
  u64 p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Read-only loads with an L2 cache policy.
__device__ __forceinline__ ulonglong2 ldg_pol(const ulonglong2 *p, u64 pol) {
  ulonglong2 r;
  asm("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
      : "=l"(r.x), "=l"(r.y)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ u64 ldg_pol(const u64 *p, u64 pol) {
  u64 r;
  asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(pol));
  return r;
}

// Asynchronous global -> shared copies (cp.async): each thread's copies form groups
// (commit), and wait<N> returns once at most the N most recent groups of this thread
// are still in flight; a barrier then makes every thread's copies visible.
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
// 16 bytes, cached in L2 only (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bulk copies by the TMA unit (cp.async.bulk, global -> shared, one instruction for a
// whole contiguous tile) completing on a shared-memory mbarrier: one thread arms the
// barrier with the byte count and issues the copy; every thread then waits on the
// barrier's phase. Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void mbar_init(u64 *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64 *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// One arrival on the barrier (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(u64 *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, u64 *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64 *bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// The slow path of mbar_wait, kept out of line (it holds the kernel's registers only
// while it runs): polls at most ~1 s of %globaltimer and 2^24 times.
static __device__ __noinline__ bool mbar_wait_slow(u64 *bar, unsigned phase) {
  const unsigned long long t0 = global_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if (global_ns() - t0 > 1000000000ull) break;
  }
  return false;
}
// Waits for phase `phase` of the barrier; false if it gave up (the caller records the
// error and carries on without the data).
__device__ __forceinline__ bool mbar_wait(u64 *bar, unsigned phase) {
  return mbar_try_wait(bar, phase) || mbar_wait_slow(bar, phase);
}

// The eight bytes of x (least significant first) as bf16 values, two per word: the
// A operand of the tensor-core basis conversion. A byte b < 256 has at most 8
// significant bits, so bf16(b) is exact: the float 2^23 + b (bits 0x4B000000 | b)
// minus 2^23 is b exactly, and its upper 16 bits are bf16(b).
__device__ __forceinline__ uint32_t bf16_of_byte(uint32_t b) {
  return __float_as_uint(__uint_as_float(0x4B000000u | b) - 8388608.0f) >> 16;
}
__device__ __forceinline__ uint4 bf16_bytes(u64 x) {
  const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
  uint4 r;
  r.x = bf16_of_byte(lo & 0xffu) | (bf16_of_byte((lo >> 8) & 0xffu) << 16);
  r.y = bf16_of_byte((lo >> 16) & 0xffu) | (bf16_of_byte(lo >> 24) << 16);
  r.z = bf16_of_byte(hi & 0xffu) | (bf16_of_byte((hi >> 8) & 0xffu) << 16);
  r.w = bf16_of_byte((hi >> 16) & 0xffu) | (bf16_of_byte(hi >> 24) << 16);
  return r;
}

// Programmatic dependent launch. Every KeySwitch kernel lets the next kernel of its
// stream launch once all its CTAs reach their end (pdl_trigger), and waits for the
// previous kernel to complete, with its memory visible, before it reads or writes any
// buffer that kernels share (pdl_wait); what comes before the wait reads only the
// context's constant tables and writes only shared memory. Without the launch
// attribute both are no-ops. (Measured on GB300: triggering at the end rather than at
// the start took (2, 2^13, 7) from 61 to 52 us per KeySwitch; triggering at the start
// slowed (2, 2^15, 10) by 16%, the dependent CTAs being placed while the previous
// kernel still ran.)
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 m) { return csub(a + b, m); }

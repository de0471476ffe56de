// tcgen05 / mbarrier helpers shared by the tensor-core kernels of the
// element strategy: bounded mbarrier waits, the K-major 128-byte-swizzle
// shared-memory descriptor, MMA issue and commit, and tensor-memory loads.
#pragma once

#include <cstdint>

namespace be {
namespace tc {

constexpr long long TIMEOUT_CYCLES = 2000000000LL;   // about one second of SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// non-blocking test of the phase (a plain try_wait may block for a
// system-dependent time, longer than a short wait limit)
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait with a suspend-time hint: the thread sleeps until the phase
// completes or about hint_ns nanoseconds pass, instead of spinning on issue
// slots that the working warps need
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns = 100000u) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
// bounded wait; false when it gave up (or another thread already did), in
// which case the abort flag is set and BE_ETIMEOUT recorded in *status.
// Between tries the thread is suspended (the suspend-time hint; the thread
// wakes when the phase completes) and the abort flag and the clock are read
// only every eighth try, so that waiting warps take few issue slots from the
// working ones.  `limit` is in SM clock cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status,
                                          long long limit = TIMEOUT_CYCLES) {
  if (mbar_test_wait(bar, parity)) return true;
  const long long start = clock64();
  if (limit < 1000000) {
    // a short limit (failure-path tests): non-blocking tests, so that the
    // limit is honoured even where a suspended try would outlast it
    while (!mbar_test_wait(bar, parity)) {
      if (*abort_flag) return false;
      if (clock64() - start > limit) {
        *abort_flag = 1;
        if (status) atomicExch(status, 9);   // BE_ETIMEOUT
        return false;
      }
    }
    return true;
  }
  const uint32_t hint = 100000u;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait_sleep(bar, parity, hint)) return true;
    if ((it & 7u) == 0u) {
      if (*abort_flag) return false;
      if (clock64() - start > limit) {
        *abort_flag = 1;
        if (status) atomicExch(status, 9);   // BE_ETIMEOUT
        return false;
      }
    }
  }
}

// make this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// the same for the 32-byte-swizzle layout: rows of 32 bytes (one K-step of
// 16 bf16), 8-row groups 256 bytes apart
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused: one swizzle atom along K)
  d |= (uint64_t)(256 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)6 << 61;                 // 32-byte swizzle
  return d;
}

// instruction descriptor of kind::f16 with D f32, A and B bf16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this thread's lane (no wait)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace be

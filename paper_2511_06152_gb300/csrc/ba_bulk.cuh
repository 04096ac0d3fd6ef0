// Bulk asynchronous copies global -> shared memory (the copy engine of
// sm_90+ / sm_100+, "cp.async.bulk") completed through a shared-memory
// mbarrier, as inline PTX.
//
// Rules kept by every caller: source and destination 16-byte aligned, sizes
// multiples of 16 bytes; the source range is rounded outward to 16 bytes
// inside an allocation whose sub-buffers start 256-byte aligned and are
// padded to 256 bytes, so the rounded range never leaves the buffer.
// Every wait is bounded: it gives up after a time limit and reports it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bagpu {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the barrier's initialisation visible to the copy engine
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of the given parity to complete; false after limit_ns
// (or 2^24 polls) without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// 16-byte rounding of a source range [p, p + bytes)
struct BulkRange {
  const char* src;   // rounded-down start
  uint32_t bytes;    // rounded-up length
  uint32_t lead;     // bytes between the rounded start and p
};

__device__ __forceinline__ BulkRange bulk_range(const void* p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = a & ~(uintptr_t)15;
  const uintptr_t hi = (a + bytes + 15) & ~(uintptr_t)15;
  return BulkRange{reinterpret_cast<const char*>(lo), static_cast<uint32_t>(hi - lo), static_cast<uint32_t>(a - lo)};
}

}  // namespace bagpu

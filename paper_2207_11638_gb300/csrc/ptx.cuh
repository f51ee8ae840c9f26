// Inline-PTX helpers: mbarriers and bulk asynchronous copies (TMA engine).
#pragma once
#include <cstdint>

namespace cdct {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async (bulk copy) proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy accesses (bulk copies into a stage that was just read)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after about `limit`
// SM cycles (the bulk copies it tracks then failed to land).  Returns false
// on time-out; the caller records the error and stops.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned); completion is reported to `bar` as transaction bytes
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 policy for data read exactly once
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ uint4 lds_v4(const void* p) {
  return *reinterpret_cast<const uint4*>(p);
}

// sign-extend the low / high 16 bits of a word (byte permute with sign replication)
__device__ __forceinline__ int sext_lo16(uint32_t u) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, 0x9910;" : "=r"(r) : "r"(u));
  return static_cast<int>(r);
}
__device__ __forceinline__ int sext_hi16(uint32_t u) {
  uint32_t r;
  asm("prmt.b32 %0, %1, 0, 0xBB32;" : "=r"(r) : "r"(u));
  return static_cast<int>(r);
}
// zero-extend byte k of a word
__device__ __forceinline__ int byte_u8(uint32_t u, int k) {
  uint32_t r;
  const uint32_t sel = 0x4440u | static_cast<uint32_t>(k);
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(u), "r"(sel));
  return static_cast<int>(r);
}

}  // namespace cdct

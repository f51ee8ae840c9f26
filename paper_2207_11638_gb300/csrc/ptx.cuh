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

// Test phase `parity`; if it is not complete the thread is suspended (not
// spinning) until it completes or about `suspend_ns` elapse.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t suspend_ns = 200000u) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after about `limit`
// SM cycles (the bulk copies it tracks then failed to land).  Returns false
// on time-out; the caller records the error and stops.
// Each try_wait suspends the warp in hardware until the phase completes or
// the hardware's own time limit passes, so the poll loop takes few issue
// slots and the warp resumes as soon as its data has landed.
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
// L2 policy of ordinary priority (data read again shortly after)
__device__ __forceinline__ uint64_t policy_evict_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// 256-bit streaming store of 8 floats (p 32-byte aligned): one full 32-byte sector per thread
__device__ __forceinline__ void stcs_v8(float* p, const float* v) {
  asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
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

namespace cdct {

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace cdct

namespace cdct {

// ---------------------------------------------------------------------------
// Packed float pairs (Blackwell f32x2 arithmetic): two IEEE single-precision
// operations per instruction, each rounded to nearest as its scalar form.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpk2(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---------------------------------------------------------------------------
// Exact integer pixels as floats without a conversion instruction.
// 0x4B400000 is 1.5 * 2^23; its low 16 bits are the integer part's low bits,
// so placing a 16-bit value there encodes 12582912 + value exactly.
// For int16 the value is stored offset by 32768 (bit 15 flipped).
// ---------------------------------------------------------------------------
constexpr float kMagicU8 = 12582912.0f;            // 1.5 * 2^23
constexpr float kMagicI16 = 12582912.0f + 32768.0f;

// low / high int16 of a word, encoded as magic floats
__device__ __forceinline__ float i16lo_magic(uint32_t u) {
  return __uint_as_float((u & 0xFFFFu) ^ 0x4B408000u);
}
__device__ __forceinline__ float i16hi_magic(uint32_t u) {
  return __uint_as_float((u >> 16) ^ 0x4B408000u);
}
// byte k of a word, encoded as a magic float
__device__ __forceinline__ float u8_magic(uint32_t u, int k) {
  uint32_t r;
  const uint32_t sel = 0x7640u | static_cast<uint32_t>(k);   // bytes: u.k, 0x00, 0x40, 0x4B
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(u), "r"(0x4B400000u), "r"(sel));
  return __uint_as_float(r);
}

// ---------------------------------------------------------------------------
// Division by a fixed 32-bit divisor: q = umulhi(n, m) is exact or one too
// small for m = floor((2^32 - 1) / d), so one correction step makes it exact
// for every n < 2^32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f, uint32_t& rem) {
  uint32_t q = __umulhi(n, f.m);
  uint32_t r = n - q * f.d;
  if (r >= f.d) { ++q; r -= f.d; }
  rem = r;
  return q;
}

}  // namespace cdct

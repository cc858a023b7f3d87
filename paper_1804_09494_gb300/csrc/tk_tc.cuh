// tcgen05 / mbarrier / bulk-copy helpers shared by the tensor-core kernels
// (inline PTX, sm_100 family).  Every wait is bounded.
#pragma once
#include <stdint.h>

namespace tk_tc {

constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (m, k) in a K-major tile with 128-byte swizzle (8-row atoms of 1 KB)
__device__ __forceinline__ uint32_t sw128_off(int m, int k) {
  const int r8 = m & 7;
  return (m >> 3) * 1024 + r8 * 128 + (((k >> 2) ^ r8) << 4) + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// kind::tf32 instruction descriptor: D FP32, A and B TF32 K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ uint32_t mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
      : "=r"(done)
      : "r"(addr), "r"(parity)
      : "memory");
  return done;
}

// One thread: wait for the phase with the given parity, bounded by kWaitCycles.
__device__ __forceinline__ bool mbar_wait(const uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  while (!mbar_try(addr, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// Whole warp (converged): the same wait with an outcome common to all lanes,
// so that the warp-collective tcgen05 instructions after it are executed by
// every lane or by none.  Bounded by kWaitCycles and, if cap > 0, by cap polls;
// cap < 0 abandons the wait at once (fault injection).
__device__ __forceinline__ bool mbar_wait_warp(const uint64_t* bar, uint32_t parity, int cap) {
  if (cap < 0) return false;
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  for (int polls = 1;; ++polls) {
    const uint32_t done = mbar_try(addr, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    const bool out = clock64() - t0 > kWaitCycles || (cap > 0 && polls >= cap);
    if (__any_sync(0xffffffffu, out)) return false;
  }
}

// bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into
// shared memory, completing on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// byte offset of element (m, k) of a K-major 16-bit tile with 64-byte swizzle
// (rows of 32 elements, 8-row atoms of 512 B; 16-byte chunk index k / 8
// XORed with address bits 7-8, i.e. (m & 7) >> 1)
__device__ __forceinline__ uint32_t sw64_off(int m, int k) {
  const int r8 = m & 7;
  return (m >> 3) * 512 + r8 * 64 + ((((k >> 3) ^ (r8 >> 1)) & 3) << 4) + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;   // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)4 << 61;            // 64-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16 K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

}  // namespace tk_tc

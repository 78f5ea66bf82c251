// tma.cuh — Tensor Memory Accelerator (TMA) loads and shared-memory mbarriers used by the
// library's staged kernels: tiled cp.async.bulk.tensor loads that complete on an mbarrier, and
// bounded waits that give up after a fixed time, set the kernel's status word to BHT_ETIMEOUT (6)
// and let the CTA wind down instead of spinning forever.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

namespace bht {
namespace tma {

constexpr uint64_t WAIT_NS = 1000000000ull;  // a wait gives up after one second

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

// Bounded wait for the completion of phase `parity` of barrier b; false after WAIT_NS (the status
// word then holds BHT_ETIMEOUT) or as soon as another thread has set the status word.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status) {
  uint32_t ok = 0;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255) {
      const uint64_t t = gtimer();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > WAIT_NS) {
        atomicExch(status, 6);
        return false;
      }
      if (*(volatile int*)status != 0) return false;
    }
  }
}

// Tiled 3-D load of one box at coordinates (x, y, z) (innermost first) into shared memory `dst`,
// completing on barrier `bar`. x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void load_3d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Offset in bytes of fp32 element c (< 32) of 128-byte row r of a tile written with
// CU_TENSOR_MAP_SWIZZLE_128B into a 1024-byte aligned buffer: the 16-byte chunks of a row are
// permuted by the row index modulo 8.
__device__ __forceinline__ uint32_t sw128_offset(uint32_t r, uint32_t c) {
  return (r << 7) + ((((c >> 2) ^ (r & 7u))) << 4) + ((c & 3u) << 2);
}

}  // namespace tma

// The driver's cuTensorMapEncodeTiled, looked up once through the runtime (nullptr when missing).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace bht

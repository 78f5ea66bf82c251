// sync.cuh — device-side reductions and the bounded grid barrier shared by the
// cooperative kernels (tridiagonalisation, Householder QR).
#pragma once
#include <cstdint>

namespace bht {

struct Barrier {
  unsigned int count;
  // written by the host before a launch (zero normally): bit 0 makes CTA 0 withhold its first arrival,
  // bits 16..31 shorten the wait limit to that many milliseconds (a test of the timeout path: every
  // CTA's wait then gives up, the status word reports BHT_ETIMEOUT and the kernel returns)
  unsigned int flags;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch on a counter that only grows (zero at launch): the k-th call
// of every CTA adds one with a release reduction, which returns nothing, and waits until the counter
// reaches k * gridDim.x. `epoch` counts the calls (the same in every thread of the CTA). The wait is
// limited to 1 s (or to the milliseconds in flags, the Barrier's flags word read once by the kernel's
// thread 0): returns false when it gave up (the status word then holds BHT_ETIMEOUT = 6) or another
// CTA reported a failure. With one CTA it is __syncthreads.
__device__ __forceinline__ bool grid_barrier_count(Barrier* bar, unsigned int& epoch, int* status,
                                                   unsigned int flags = 0u) {
  __shared__ int ok;
  __syncthreads();
  if (gridDim.x == 1) return true;
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned int target = epoch * gridDim.x;
    const uint64_t limit = (flags >> 16) ? (uint64_t)(flags >> 16) * 1000000ull : 1000000000ull;
    if (!((flags & 1u) && blockIdx.x == 0 && epoch == 1))
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->count) : "memory");
    const uint64_t t0 = global_ns();
    unsigned int cur;
    for (uint32_t spin = 0;; ++spin) {
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((int)(cur - target) >= 0) break;
      if ((spin & 63) == 63) {
        if (*(volatile int*)status != 0) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > limit) {
          atomicExch(status, 6);
          ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the first `n` lanes' values (n <= 32) in log2(n) rounded up shuffle steps; lanes beyond n
// must hold 0. Every lane of the group of the first `span` lanes gets the sum.
__device__ __forceinline__ double warp_sum_first(double v, int n) {
  int span = 1;
  while (span < n) span <<= 1;
  for (int o = span >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (every thread gets the result); red holds 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    // second level over the warps' partial sums only: log2 of the warp count rounded up, not 5 steps
    const int nwarps = (int)(blockDim.x >> 5);
    double t = (l < nwarps) ? red[l] : 0.0;
    int span = 1;
    while (span < nwarps) span <<= 1;
    for (int o = span >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (l == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

}  // namespace bht

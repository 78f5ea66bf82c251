// sync.cuh — device-side reductions and the bounded grid barrier shared by the
// cooperative kernels (tridiagonalisation, Householder QR).
#pragma once
#include <cstdint>

namespace bht {

struct Barrier {
  unsigned int count;
  unsigned int gen;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch with a 1 s limit: arrival is a
// release add on the counter, the last CTA resets it and publishes the next
// generation with a release store, the others poll the generation with
// acquire loads. Returns false when the wait gave up (the status word then
// holds BHT_ETIMEOUT = 6) or another CTA reported a failure. With one CTA it
// is __syncthreads.
__device__ __forceinline__ bool grid_barrier(Barrier* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (gridDim.x == 1) return true;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned int g, arrived;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(g) : "l"(&bar->gen) : "memory");
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&bar->count) : "memory");
    if (arrived == gridDim.x - 1) {
      asm volatile("st.relaxed.gpu.u32 [%0], 0;" ::"l"(&bar->count) : "memory");
      asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(&bar->gen), "r"(g + 1) : "memory");
    } else {
      const uint64_t t0 = global_ns();
      unsigned int cur;
      for (uint32_t spin = 0;; ++spin) {
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->gen) : "memory");
        if (cur != g) break;
        if ((spin & 63) == 63) {
          if (*(volatile int*)status != 0) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > 1000000000ull) {
            atomicExch(status, 6);
            ok = 0;
            break;
          }
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

// Sum over the block (every thread gets the result); red holds 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

}  // namespace bht

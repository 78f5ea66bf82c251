// probe.cu — measured FMA throughput of this GPU, the denominator of the ALU rooflines reported for
// the FP64 node linear algebra and the FP32 SIMT kernels. Every thread runs eight independent FMA
// chains (enough to cover the pipe latency), every SM gets the same number of resident CTAs, and the
// launch is timed with CUDA events on the caller's stream after a warm-up launch.
#include <algorithm>

#include "bht.h"
#include "internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(int64_t iters, T seed, T* __restrict__ sink) {
  T a[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = seed + (T)(threadIdx.x + c);
  const T m = (T)0.999999, k = (T)1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) a[c] = fma(a[c], m, k);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += a[c];
  if (s == (T)-1.2345) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

bht_status set_error(bht_status st, const char* msg) {
  bht::set_last_error(msg);
  return st;
}

template <typename T>
cudaError_t run_probe(int64_t iters, int grid, T* sink, cudaStream_t s, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<grid, PROBE_THREADS, 0, s>>>(iters / 8 + 1, (T)1, sink);  // warm-up
    bht::note_launch();
    e = cudaEventRecord(e0, s);
  }
  if (e == cudaSuccess) {
    fma_probe_kernel<T><<<grid, PROBE_THREADS, 0, s>>>(iters, (T)1, sink);
    bht::note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" bht_status bht_probe_fma_rate(int32_t dtype, double* tflops, void* stream) {
  if (!tflops || (dtype != BHT_F32 && dtype != BHT_F64)) return set_error(BHT_EINVAL, "bad argument");
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = dtype == BHT_F64
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<double>, PROBE_THREADS, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<float>, PROBE_THREADS, 0);
  if (e != cudaSuccess || per_sm < 1 || nsm < 1) {
    cudaGetLastError();
    return set_error(BHT_ECUDA, "occupancy query failed");
  }
  const int grid = nsm * per_sm;
  // about 10 ms of work at the nominal rates (FP64 1.25 TFLOP/s, FP32 80 TFLOP/s)
  const double target_flops = (dtype == BHT_F64 ? 1.25e12 : 8.0e13) * 0.01;
  const int64_t iters =
      std::max<int64_t>(64, (int64_t)(target_flops / (2.0 * PROBE_CHAINS * (double)grid * PROBE_THREADS)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* sink = nullptr;
  e = cudaMallocAsync(&sink, sizeof(double) * grid, s);
  float ms = 0.f;
  if (e == cudaSuccess)
    e = dtype == BHT_F64 ? run_probe<double>(iters, grid, static_cast<double*>(sink), s, &ms)
                         : run_probe<float>(iters, grid, static_cast<float*>(sink), s, &ms);
  if (sink) {
    const cudaError_t ef = cudaFreeAsync(sink, s);
    if (e == cudaSuccess) e = ef;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || !(ms > 0.f)) {
    cudaGetLastError();
    return set_error(BHT_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "probe took no time");
  }
  *tflops = 2.0 * PROBE_CHAINS * (double)iters * (double)grid * PROBE_THREADS / (ms * 1e-3) / 1e12;
  return BHT_OK;
}

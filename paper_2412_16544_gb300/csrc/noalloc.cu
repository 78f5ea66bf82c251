// noalloc.cu — bht_mode_product_noalloc: the tensor-core mode product of the
// innermost axis with its scratch (the split TF32 weight planes and the
// device status word) in a file-scope device array instead of memory from
// cudaMalloc / the stream-ordered pool.
//
// Who needs it: callers that may not allocate device memory at the time of
// the call, e.g. an application whose device memory is owned by another
// allocator (a framework's caching allocator that has reserved the GPU), or a
// latency-critical loop where cudaMalloc / cudaFree could synchronise the
// device or take an unbounded time. They pass inputs and outputs they own;
// the library keeps nothing else.
//
// The array holds NOALLOC_SCRATCH_BYTES on every GPU that loads the library,
// until the process exits. Its device address is looked up once per device
// (cudaGetSymbolAddress with that device current) on the first call made on
// that device; make that first call before any stream capture. All calls
// share the one array and it keeps the last call's contents: calls that
// overlap on the GPU (on different streams, or from several host threads)
// race on it and must be serialised by the caller.
#include <mutex>

#include "bht.h"
#include "internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_K = 512;   // contracted extent
constexpr int64_t NOALLOC_MAX_S = 256;   // output extent
constexpr size_t NOALLOC_STATUS_BYTES = 256;
// two weight planes [S_pad][K_pad] fp32 at the maximum sizes, then the status word
constexpr size_t NOALLOC_SCRATCH_BYTES = 2 * NOALLOC_MAX_S * NOALLOC_MAX_K * sizeof(float) + NOALLOC_STATUS_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {};

bht_status set_error(bht_status st, const char* msg) {
  bht::set_last_error(msg);  // read back with bht_last_error()
  return st;
}

// Device (or managed) memory, by the pointer's attributes: a query that allocates nothing. A host
// pointer handed to the tensor map or to the kernels would be a fault instead of an error code.
bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" bht_status bht_mode_product_noalloc(const float* X, int64_t rows, int64_t K, const double* U, int64_t S,
                                               float* out, int64_t R2, double* norms, void* stream) {
  if (!X || !U || !out) return set_error(BHT_EINVAL, "null argument");
  if (rows < 1 || K < 1 || S < 1 || R2 < 1 || rows % R2 != 0)
    return set_error(BHT_EINVAL, "bad sizes (rows must be a multiple of R2)");
  if (K % 4 != 0) return set_error(BHT_EINVAL, "K must be a multiple of 4 (tensor-map row pitch)");
  if (!on_device(X) || !on_device(U) || !on_device(out) || (norms && !on_device(norms)))
    return set_error(BHT_EINVAL, "bht_mode_product_noalloc takes device pointers (X, U, out, norms)");
  if (K > NOALLOC_MAX_K || S > NOALLOC_MAX_S)
    return set_error(BHT_ECAPACITY, "bht_mode_product_noalloc: K > 512 or S > 256 exceeds its static scratch");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    cudaGetLastError();
    return set_error(BHT_ECUDA, "no current CUDA device");
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return set_error(BHT_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* W = static_cast<float*>(base);
  int* status = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + NOALLOC_SCRATCH_BYTES -
                                       NOALLOC_STATUS_BYTES);
  // the status word must start at zero; the weight planes are rewritten in full (zero padded) every call
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = bht::launch_prep_tc_weights(U, K, S, S, true, W, 2, s);
  if (e == cudaSuccess)
    e = bht::launch_ttm_tc(X, rows, K, W, S, 2, out, R2, norms, norms ? norms + 1 : nullptr, status, s);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(BHT_ECUDA, cudaGetErrorString(e));
  }
  if (h) return set_error((bht_status)h, "a bounded device-side wait gave up (tensor-core pipeline)");
  return BHT_OK;
}

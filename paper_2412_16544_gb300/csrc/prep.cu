// prep.cu — data preparation around the method and the error of unseen items:
//   * per-group normalisation of the snapshots (maximum absolute value, unit vector, z-score; the
//     scientific-data experiments normalise every physical quantity of every simulation on its own);
//   * a permutation of the item axes (the axis-ordering study of App. D);
//   * per-item squared errors, from which the relative test error (eq. generalization_performance)
//     averages the per-item relative errors.
// All of these are single passes over HBM: grid-stride loops, FP64 accumulation, one atomic per block.
#include <algorithm>
#include <cmath>

#include "bht.h"
#include "internal.cuh"
#include "sync.cuh"

namespace bht {
namespace {

constexpr int NT = 256;
constexpr int64_t CHUNK = 8192;  // elements of one group handled by one block

template <typename T>
__device__ __forceinline__ double ld(const T* p, int64_t i) {
  return static_cast<double>(p[i]);
}

// Flattened grid: block b covers elements [c * CHUNK, (c + 1) * CHUNK) of group b / chunks. Sums of y,
// of y^2 and the largest |y| of every group: stats[3g], stats[3g + 1], stats[3g + 2] (the maximum is
// kept as the bit pattern of a non-negative double, whose integer order is the numeric order).
template <typename T>
__global__ void group_stats_kernel(const T* __restrict__ Y, int64_t size, int64_t chunks, double* __restrict__ stats) {
  __shared__ double red[33];
  const int64_t g = blockIdx.x / chunks, c = blockIdx.x % chunks;
  const T* y = Y + g * size;
  const int64_t lo = c * CHUNK, hi = min(size, lo + CHUNK);
  double s = 0.0, s2 = 0.0, m = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const double v = ld(y, i);
    s += v;
    s2 = fma(v, v, s2);
    m = fmax(m, fabs(v));
  }
  s = block_sum(s, red);
  s2 = block_sum(s2, red);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double mx[32];
  if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) m = fmax(m, mx[w]);
    atomicAdd(&stats[3 * g], s);
    atomicAdd(&stats[3 * g + 1], s2);
    atomicMax(reinterpret_cast<unsigned long long*>(&stats[3 * g + 2]),
              static_cast<unsigned long long>(__double_as_longlong(m)));
  }
}

// Second pass of the z-score: sum of (y - mean)^2 into cen[g] (no cancellation against the mean).
template <typename T>
__global__ void group_centred_kernel(const T* __restrict__ Y, int64_t size, int64_t chunks,
                                     const double* __restrict__ stats, double* __restrict__ cen) {
  __shared__ double red[33];
  const int64_t g = blockIdx.x / chunks, c = blockIdx.x % chunks;
  const T* y = Y + g * size;
  const double mu = stats[3 * g] / (double)size;
  const int64_t lo = c * CHUNK, hi = min(size, lo + CHUNK);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const double v = ld(y, i) - mu;
    s = fma(v, v, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) atomicAdd(&cen[g], s);
}

// shift and scale of every group; a scale that is zero or not finite becomes 1 (the group is only
// shifted), so that a constant snapshot stays finite.
__global__ void group_params_kernel(const double* __restrict__ stats, const double* __restrict__ cen, int64_t groups,
                                    int64_t size, int kind, double* __restrict__ params) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= groups) return;
  double shift = 0.0, scale = 1.0;
  if (kind == 1) {
    scale = stats[3 * g + 2];
  } else if (kind == 2) {
    scale = sqrt(stats[3 * g + 1]);
  } else if (kind == 3) {
    shift = stats[3 * g] / (double)size;
    scale = sqrt(cen[g] / (double)size);
  }
  if (!(scale > 0.0) || !isfinite(scale)) scale = 1.0;
  params[2 * g] = shift;
  params[2 * g + 1] = scale;
}

template <typename T>
__global__ void group_apply_kernel(T* __restrict__ Y, int64_t size, int64_t chunks, const double* __restrict__ params,
                                   int inverse) {
  const int64_t g = blockIdx.x / chunks, c = blockIdx.x % chunks;
  T* y = Y + g * size;
  const double shift = params[2 * g], scale = params[2 * g + 1];
  const int64_t lo = c * CHUNK, hi = min(size, lo + CHUNK);
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const double v = ld(y, i);
    y[i] = static_cast<T>(inverse ? fma(v, scale, shift) : (v - shift) / scale);
  }
}

struct PermArgs {
  int d;
  int64_t out_dims[16];
  int64_t in_stride[16];  // stride in the input item of the axis that lands at output position k
};

template <typename T>
__global__ void permute_items_kernel(const T* __restrict__ Y, T* __restrict__ out, int64_t total, int64_t item,
                                     PermArgs a) {
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = o / item;
    int64_t r = o - n * item, src = 0;
    for (int k = a.d - 1; k >= 0; --k) {
      const int64_t q = r / a.out_dims[k];
      src += (r - q * a.out_dims[k]) * a.in_stride[k];
      r = q;
    }
    out[o] = Y[n * item + src];
  }
}

template <typename T>
__global__ void item_errors_kernel(const T* __restrict__ X, const double* __restrict__ Xh, int64_t item,
                                   int64_t chunks, double* __restrict__ err2, double* __restrict__ nrm2) {
  __shared__ double red[33];
  const int64_t n = blockIdx.x / chunks, c = blockIdx.x % chunks;
  const int64_t lo = c * CHUNK, hi = min(item, lo + CHUNK);
  const T* x = X + n * item;
  const double* xh = Xh + n * item;
  double e = 0.0, s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += NT) {
    const double v = ld(x, i), dv = v - xh[i];
    e = fma(dv, dv, e);
    s = fma(v, v, s);
  }
  e = block_sum(e, red);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    atomicAdd(&err2[n], e);
    atomicAdd(&nrm2[n], s);
  }
}

int64_t chunks_of(int64_t size) { return (size + CHUNK - 1) / CHUNK; }

}  // namespace

cudaError_t launch_normalize(void* Y, int dtype, int64_t groups, int64_t size, int kind, double* params,
                             cudaStream_t s) {
  if (groups <= 0 || size <= 0) return cudaSuccess;
  const int64_t ch = chunks_of(size), blocks = groups * ch;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  double* stats = nullptr;
  cudaError_t e = cudaMallocAsync(&stats, sizeof(double) * 4 * groups, s);
  if (e != cudaSuccess) return e;
  double* cen = stats + 3 * groups;
  e = cudaMemsetAsync(stats, 0, sizeof(double) * 4 * groups, s);
  {
    ProfScope prof(K_PREP, s, 3.0 * (double)groups * (double)size,
                   (double)groups * (double)size * (dtype == BHT_F64 ? 8.0 : 4.0));
    if (e == cudaSuccess && kind != 0) {
      if (dtype == BHT_F64)
        group_stats_kernel<double><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const double*>(Y), size, ch, stats);
      else
        group_stats_kernel<float><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const float*>(Y), size, ch, stats);
      note_launch();
      if (kind == 3) {
        if (dtype == BHT_F64)
          group_centred_kernel<double><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const double*>(Y), size, ch, stats,
                                                                      cen);
        else
          group_centred_kernel<float><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const float*>(Y), size, ch, stats,
                                                                     cen);
        note_launch();
      }
    }
  }
  if (e == cudaSuccess) {
    group_params_kernel<<<(unsigned)((groups + 255) / 256), 256, 0, s>>>(stats, cen, groups, size, kind, params);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && kind != 0) {
    ProfScope prof(K_PREP, s, 2.0 * (double)groups * (double)size,
                   2.0 * (double)groups * (double)size * (dtype == BHT_F64 ? 8.0 : 4.0));
    if (dtype == BHT_F64)
      group_apply_kernel<double><<<(unsigned)blocks, NT, 0, s>>>(static_cast<double*>(Y), size, ch, params, 0);
    else
      group_apply_kernel<float><<<(unsigned)blocks, NT, 0, s>>>(static_cast<float*>(Y), size, ch, params, 0);
    note_launch();
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(stats, s);
  return e != cudaSuccess ? e : f;
}

cudaError_t launch_denormalize(void* Y, int dtype, int64_t groups, int64_t size, const double* params,
                               cudaStream_t s) {
  if (groups <= 0 || size <= 0) return cudaSuccess;
  const int64_t ch = chunks_of(size), blocks = groups * ch;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  ProfScope prof(K_PREP, s, 2.0 * (double)groups * (double)size,
                 2.0 * (double)groups * (double)size * (dtype == BHT_F64 ? 8.0 : 4.0));
  if (dtype == BHT_F64)
    group_apply_kernel<double><<<(unsigned)blocks, NT, 0, s>>>(static_cast<double*>(Y), size, ch, params, 1);
  else
    group_apply_kernel<float><<<(unsigned)blocks, NT, 0, s>>>(static_cast<float*>(Y), size, ch, params, 1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_permute_items(const void* Y, int dtype, int64_t N, int d, const int64_t* dims, const int* perm,
                                 void* out, cudaStream_t s) {
  if (d < 1 || d > 16) return cudaErrorInvalidValue;
  PermArgs a;
  a.d = d;
  int64_t in_stride[16];
  int64_t item = 1;
  for (int k = d - 1; k >= 0; --k) {
    in_stride[k] = item;
    item *= dims[k];
  }
  for (int k = 0; k < d; ++k) {
    a.out_dims[k] = dims[perm[k]];
    a.in_stride[k] = in_stride[perm[k]];
  }
  const int64_t total = N * item;
  if (total <= 0) return cudaSuccess;
  ProfScope prof(K_PREP, s, 0.0, 2.0 * (double)total * (dtype == BHT_F64 ? 8.0 : 4.0));
  const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  if (dtype == BHT_F64)
    permute_items_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(Y), static_cast<double*>(out), total,
                                                      item, a);
  else
    permute_items_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(Y), static_cast<float*>(out), total,
                                                     item, a);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_item_errors(const void* X, int dtype, const double* Xh, int64_t N, int64_t item, double* err2,
                               double* nrm2, cudaStream_t s) {
  if (N <= 0 || item <= 0) return cudaSuccess;
  const int64_t ch = chunks_of(item), blocks = N * ch;
  if (blocks > 2147483647LL) return cudaErrorInvalidValue;
  ProfScope prof(K_PREP, s, 4.0 * (double)N * (double)item,
                 (double)N * (double)item * ((dtype == BHT_F64 ? 8.0 : 4.0) + 8.0));
  if (dtype == BHT_F64)
    item_errors_kernel<double><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const double*>(X), Xh, item, ch, err2, nrm2);
  else
    item_errors_kernel<float><<<(unsigned)blocks, NT, 0, s>>>(static_cast<const float*>(X), Xh, item, ch, err2, nrm2);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

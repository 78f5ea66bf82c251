// synth.cu — device generator of the smooth sensor-grid stream (sums of separable products of random
// Chebyshev series plus Gaussian noise), so that a long stream can be drawn straight into HBM at the
// rate it is compressed instead of being built on the host and copied.
//
//   item[i_1..i_d] = sum_{q < terms} prod_{m < d} f_{qm}(i_m) + noise_std * z(item, flat index),
//   f_{qm}(i)      = sum_{j <= degree} c[q][m][j] T_j(x_i),  x_i = -1 + 2 i / (n - 1),
//
// with T_j the Chebyshev polynomials (three-term recurrence), c the caller's coefficients and z a
// counter-based normal draw: the item's base word b = mix64(seed * 2^32 + item), word k =
// mix64(b + (k + 1) * gamma) (the k-th output of a SplitMix64 sequence from b; Steele, Lea and Flood,
// OOPSLA 2014), and the Box-Muller transform of two 24-bit uniforms of word k gives elements 2k
// (cosine) and 2k + 1 (sine). This is input synthesis, not part of the decomposition.
#include <algorithm>
#include <cmath>

#include "bht.h"
#include "internal.cuh"

namespace {

constexpr int SYNTH_MAX_TERMS = 64;
constexpr int SYNTH_MAX_N = 64;
constexpr int SYNTH_MAX_D = 8;
constexpr int SYNTH_MAX_DEGREE = 32;
constexpr int SYNTH_THREADS = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// f[item][q][m][i] (fp32) from the coefficients c[item][q][m][j] (fp64), one thread per value.
__global__ void cheb_factor_kernel(const double* __restrict__ c, int64_t count, int terms, int d, int degree, int n,
                                   float* __restrict__ f) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = count * terms * d * n;
  if (t >= total) return;
  const int i = (int)(t % n);
  const int64_t qm = t / n;  // (item * terms + q) * d + m
  const double x = (n > 1) ? -1.0 + 2.0 * (double)i / (double)(n - 1) : 0.0;
  const double* cc = c + qm * (degree + 1);
  double tm = 1.0, tj = x, acc = cc[0];
  if (degree >= 1) acc = fma(cc[1], x, acc);
  for (int j = 2; j <= degree; ++j) {
    const double tn = 2.0 * x * tj - tm;
    acc = fma(cc[j], tn, acc);
    tm = tj;
    tj = tn;
  }
  f[t] = (float)acc;
}

// The uniforms (k + 1/2) 2^-24 of two 24-bit integers k, formed in FP32 (k 2^-24 is exact; adding 2^-25
// rounds to even only for k >= 2^23, a change of at most 2^-25), then the Box-Muller pair.
__device__ __forceinline__ void noise_pair(uint64_t base, int64_t word, float sd, float& z0, float& z1) {
  const uint64_t w = mix64(base + ((uint64_t)word + 1ull) * 0x9E3779B97F4A7C15ull);
  const float u1 = fmaf((float)(uint32_t)(w >> 40), 0x1p-24f, 0x1p-25f);
  const float u2 = fmaf((float)(uint32_t)((w >> 8) & 0xFFFFFFull), 0x1p-24f, 0x1p-25f);
  const float r = sd * sqrtf(-2.f * logf(u1));
  float sn, cs;
  sincospif(2.f * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

// One block per (item, chunk of slabs); a slab is the n x n plane of the last two modes for one index of
// the first d - 2 modes. The factors of the last two modes stay in shared memory for the block, and the
// product over the first d - 2 modes is formed once per slab and term. With n % 8 == 0 a thread makes
// 8 consecutive elements of a row (one factor product per term, one noise word per two elements, two
// 16-byte stores); otherwise one element at a time.
template <bool OCTETS>
__global__ void __launch_bounds__(SYNTH_THREADS) cheb_items_kernel(const float* __restrict__ f, int terms, int d,
                                                                  int n, int64_t slabs, int64_t slabs_per_block,
                                                                  double noise_std, uint64_t seed,
                                                                  int64_t first_item, float* __restrict__ out) {
  __shared__ __align__(16) float fa[SYNTH_MAX_TERMS * SYNTH_MAX_N];
  __shared__ __align__(16) float fb[SYNTH_MAX_TERMS * SYNTH_MAX_N];
  __shared__ float Pall[SYNTH_MAX_N * SYNTH_MAX_TERMS];  // [slab of the block][term]
  const int64_t item = blockIdx.y;
  const float* fi = f + item * (int64_t)terms * d * n;  // [terms][d][n]
  for (int t = threadIdx.x; t < terms * n; t += blockDim.x) {
    const int q = t / n, i = t % n;
    fa[t] = fi[((int64_t)q * d + (d - 2)) * n + i];
    fb[t] = fi[((int64_t)q * d + (d - 1)) * n + i];
  }
  const int64_t nn = (int64_t)n * n;
  const int64_t per_item = slabs * nn;
  const uint64_t base = mix64((seed << 32) + (uint64_t)(first_item + item));
  const float sd = (float)noise_std;
  float* o = out + item * per_item;
  const int64_t s0 = blockIdx.x * slabs_per_block, s1 = min(slabs, s0 + slabs_per_block);
  // the products over the first d - 2 modes of every slab of the block, once
  for (int t = threadIdx.x; t < (int)(s1 - s0) * terms; t += blockDim.x) {
    const int sl_rel = t / terms, q = t - sl_rel * terms;
    float p = 1.f;
    int64_t rem = s0 + sl_rel;
    for (int m = d - 3; m >= 0; --m) {
      const int im = (int)(rem % n);
      rem /= n;
      p *= fi[((int64_t)q * d + m) * n + im];
    }
    Pall[sl_rel * terms + q] = p;
  }
  __syncthreads();
  for (int64_t sl = s0; sl < s1; ++sl) {
    const float* P = Pall + (sl - s0) * terms;
    if (OCTETS) {
      const int per_row = n / 8;
      for (int t = threadIdx.x; t < n * per_row; t += blockDim.x) {
        const int ia = t / per_row, ib0 = (t - ia * per_row) * 8;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
        for (int q = 0; q < terms; ++q) {
          const float pa = P[q] * fa[q * n + ia];
          const float4 b0 = *reinterpret_cast<const float4*>(fb + q * n + ib0);
          const float4 b1 = *reinterpret_cast<const float4*>(fb + q * n + ib0 + 4);
          v[0] = fmaf(pa, b0.x, v[0]);
          v[1] = fmaf(pa, b0.y, v[1]);
          v[2] = fmaf(pa, b0.z, v[2]);
          v[3] = fmaf(pa, b0.w, v[3]);
          v[4] = fmaf(pa, b1.x, v[4]);
          v[5] = fmaf(pa, b1.y, v[5]);
          v[6] = fmaf(pa, b1.z, v[6]);
          v[7] = fmaf(pa, b1.w, v[7]);
        }
        const int64_t E = sl * nn + (int64_t)ia * n + ib0;  // even: a row starts at a multiple of 8
        if (sd != 0.f) {
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            float z0, z1;
            noise_pair(base, (E >> 1) + u / 2, sd, z0, z1);
            v[u] += z0;
            v[u + 1] += z1;
          }
        }
        float4* dst = reinterpret_cast<float4*>(o + E);
        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
      }
    } else {
      for (int64_t e = threadIdx.x; e < nn; e += blockDim.x) {
        const int ia = (int)(e / n), ib = (int)(e % n);
        float v = 0.f;
        for (int q = 0; q < terms; ++q) v = fmaf(P[q] * fa[q * n + ia], fb[q * n + ib], v);
        const int64_t E = sl * nn + e;  // flat index within the item
        if (sd != 0.f) {
          float z0, z1;
          noise_pair(base, E >> 1, 1.f, z0, z1);
          v = fmaf(sd, (E & 1) ? z1 : z0, v);
        }
        o[E] = v;
      }
    }
  }
}

bht_status set_error(bht_status st, const char* msg) {
  bht::set_last_error(msg);
  return st;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" bht_status bht_synth_chebyshev(const double* coeffs, int64_t count, int32_t n, int32_t d, int32_t terms,
                                          int32_t degree, double noise_std, uint64_t seed, int64_t first_item,
                                          float* out, void* stream) {
  if (count == 0) return BHT_OK;
  if (!coeffs || !out || count < 0) return set_error(BHT_EINVAL, "null argument or negative count");
  if (n < 1 || n > SYNTH_MAX_N || d < 2 || d > SYNTH_MAX_D || terms < 1 || terms > SYNTH_MAX_TERMS || degree < 0 ||
      degree > SYNTH_MAX_DEGREE || count > 65535 || first_item < 0 || !(noise_std >= 0.0))
    return set_error(BHT_EINVAL,
                     "bht_synth_chebyshev: n in 1..64, d in 2..8, terms in 1..64, degree in 0..32, "
                     "count <= 65535, first_item >= 0, noise_std >= 0");
  if (!on_device(out)) return set_error(BHT_EINVAL, "bht_synth_chebyshev writes device memory");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nc = count * terms * d * (int64_t)(degree + 1);
  const int64_t nf = count * terms * d * (int64_t)n;
  cudaError_t e = cudaSuccess;
  double* dc = nullptr;
  float* df = nullptr;
  const bool host_c = !on_device(coeffs);
  e = cudaMallocAsync(reinterpret_cast<void**>(&df), sizeof(float) * nf, s);
  if (e == cudaSuccess && host_c) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&dc), sizeof(double) * nc, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, coeffs, sizeof(double) * nc, cudaMemcpyHostToDevice, s);
  }
  const double* cptr = host_c ? dc : coeffs;
  if (e == cudaSuccess) {
    bht::ProfScope ps(bht::K_PREP, s);
    cheb_factor_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(cptr, count, terms, d, degree, n, df);
    e = cudaGetLastError();
    bht::note_launch();
  }
  if (e == cudaSuccess) {
    int64_t slabs = 1;
    for (int m = 0; m < d - 2; ++m) slabs *= n;
    const int64_t spb = std::max<int64_t>(1, std::min<int64_t>(n, slabs));  // one index of mode d-3 per block
    const int64_t chunks = (slabs + spb - 1) / spb;
    if (chunks > 0x7fffffffll) {
      e = cudaErrorInvalidValue;
    } else {
      const double bytes = 4.0 * (double)count * (double)slabs * n * n;
      bht::ProfScope ps(bht::K_PREP, s, 0.0, bytes);
      dim3 grid((unsigned)chunks, (unsigned)count);
      if (n % 8 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0)
        cheb_items_kernel<true><<<grid, SYNTH_THREADS, 0, s>>>(df, terms, d, n, slabs, spb, noise_std, seed,
                                                                first_item, out);
      else
        cheb_items_kernel<false><<<grid, SYNTH_THREADS, 0, s>>>(df, terms, d, n, slabs, spb, noise_std, seed,
                                                                 first_item, out);
      e = cudaGetLastError();
      bht::note_launch();
    }
  }
  // every stream-ordered free is enqueued even after a failure, so nothing leaks
  const cudaError_t e1 = df ? cudaFreeAsync(df, s) : cudaSuccess;
  const cudaError_t e2 = dc ? cudaFreeAsync(dc, s) : cudaSuccess;
  if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
  if (e == cudaSuccess && host_c) e = cudaStreamSynchronize(s);  // the host coefficients are read by the copy
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? BHT_ENOMEM : BHT_ECUDA, cudaGetErrorString(e));
  }
  return BHT_OK;
}

// tc.cu — tcgen05 tensor-core mode product over the innermost axis.
//
//   out[(o * S + s) * R2 + i] = sum_k X[o * R2 + i][k] * U[k][s]
//
// X is an item-major layer intermediate viewed as rows of its innermost axis
// (K contiguous); U is a node basis, so this is the leaf contraction
// C x_j U_j^T of eq. ht_leaf_contraction (and of Step 1 of Algorithm 2) for
// the innermost axis j. The new axis of size S is written in front of the
// last R2-sized group of axes: R2 = 1 keeps it innermost, R2 = (product of
// all other axes) rotates it to the front, which makes the next axis the
// innermost one.
//
// Arithmetic: X is split into x_hi + x_lo with x_hi = x with its 13 low
// mantissa bits cleared (what the TF32 datapath reads) and x_lo = x - x_hi;
// U^T is rounded to TF32 (round-to-nearest), optionally with its own low part.
// Two (or three) TF32 MMAs per K step, FP32 accumulation in TMEM: the result
// carries no truncation bias and a relative error of about 2^-12 (2^-20 with
// the low part of U), which keeps the norm difference of the skip test of
// Algorithm 2 (eq. relative_error_threshold) unbiased.
//
// Structure: persistent CTAs (one per SM), 128-row tiles, 8 warps:
//   warp 0      TMA producer (cp.async.bulk.tensor, 128B swizzle)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2-3   split x into hi / lo in shared memory, fold ||X||^2 (FP64)
//   warps 4-7   epilogue: tcgen05.ld, scattered store, fold ||out||^2 (FP64)
// Every mbarrier wait is bounded (1 s); a wait that gives up sets the status
// word to BHT_ETIMEOUT and the CTA winds down.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"
#include "tcgen.cuh"
#include "tma.cuh"

namespace bht {

namespace {

constexpr int TC_THREADS = 256;
constexpr int BM = 128;           // rows per tile (MMA M)
constexpr int KC = 32;            // fp32 per 128-byte swizzle row (one K chunk)
constexpr int CHUNK_BYTES = BM * KC * 4;  // 16 KB

using tma::gtimer;
using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait;
using tma::smem_u32;

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

using tcg::fence_after;
using tcg::fence_before;
using tcg::mbar_arrive;
using tcg::mma_commit;
using tcg::mma_tf32;
using tcg::sw128_desc;
using tcg::tmem_ld16;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct TcParams {
  int64_t rows;    // rows of X
  int nkc;         // K chunks of 32
  int S;           // computed output columns
  int S_store;     // stored output columns (the first S_store); the squares of the rest go to resid
  int S_pad;       // rows of one weight plane (multiple of 16)
  int S_tile;      // MMA N per work unit (multiple of 16, <= 256)
  int n_ntiles;    // ceil(S_pad / S_tile)
  int nb;          // 1: B rounded to TF32; 2: B = hi + lo
  int nslot;       // K-chunk ring depth
  int64_t R2;      // placement of the new axis
  float* out;
  double* norm_in;
  double* norm_out;
  double* resid;
  int* status;
};

// Work unit u = (m tile, n tile): m = u / n_ntiles, n = u % n_ntiles. Every
// K chunk of a unit fills one ring slot: the X chunk (16 KB), its low part
// (16 KB) and the matching chunk of every weight plane (S_tile x 128 B each).
__global__ void __launch_bounds__(TC_THREADS, 1) ttm_tc_kernel(const __grid_constant__ CUtensorMap mapX,
                                                                const __grid_constant__ CUtensorMap mapW,
                                                                const TcParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int w_bytes = P.S_tile * 128;
  const int slot_bytes = 2 * CHUNK_BYTES + P.nb * w_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)P.nslot * slot_bytes);
  uint64_t* full = bars;                  // nslot
  uint64_t* ready = bars + P.nslot;       // nslot
  uint64_t* empty = bars + 2 * P.nslot;   // nslot
  uint64_t* tfull = bars + 3 * P.nslot;   // 2
  uint64_t* tempty = tfull + 2;           // 2
  __shared__ uint32_t tmem_base;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nunits = ((P.rows + BM - 1) / BM) * P.n_ntiles;
  const uint32_t ncols = (2 * P.S_tile <= 32) ? 32u
                         : (2 * P.S_tile <= 64) ? 64u
                         : (2 * P.S_tile <= 128) ? 128u
                         : (2 * P.S_tile <= 256) ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int i = 0; i < P.nslot; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&ready[i], 2);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    tma::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t g = 0;
      for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int64_t mt = u / P.n_ntiles;
        const int nt = (int)(u - mt * P.n_ntiles);
        for (int kc = 0; kc < P.nkc; ++kc, ++g) {
          const uint32_t slot = g % P.nslot, ph = (g / P.nslot) & 1;
          if (!mbar_wait(&empty[slot], ph ^ 1, P.status)) goto producer_done;
          uint8_t* sb = base + (size_t)slot * slot_bytes;
          mbar_expect_tx(&full[slot], (uint32_t)(CHUNK_BYTES + P.nb * w_bytes));
          tma_load_2d(&mapX, &full[slot], sb, kc * KC, (int)(mt * BM));
          for (int b = 0; b < P.nb; ++b)
            tma_load_2d(&mapW, &full[slot], sb + 2 * CHUNK_BYTES + b * w_bytes, kc * KC, b * P.S_pad + nt * P.S_tile);
        }
      }
    producer_done:;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(P.S_tile >> 3) << 17) |
                             ((uint32_t)(BM >> 4) << 24);
      bool ok = true;
      uint32_t g = 0, it = 0;
      for (int64_t u = blockIdx.x; ok && u < nunits; u += gridDim.x, ++it) {
        const uint32_t acc = it & 1, aph = (it >> 1) & 1;
        if (!mbar_wait(&tempty[acc], aph ^ 1, P.status)) break;
        fence_after();
        const uint32_t dt = tmem + acc * P.S_tile;
        for (int kc = 0; kc < P.nkc; ++kc, ++g) {
          const uint32_t slot = g % P.nslot, ph = (g / P.nslot) & 1;
          if (!mbar_wait(&full[slot], ph, P.status) || !mbar_wait(&ready[slot], ph, P.status)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sb = smem_u32(base + (size_t)slot * slot_bytes);
          const uint32_t ahi = sb, alo = sb + CHUNK_BYTES, bhi = sb + 2 * CHUNK_BYTES, blo = bhi + w_bytes;
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {
            const uint64_t bd = sw128_desc(bhi + 32 * k4);
            mma_tf32(dt, sw128_desc(ahi + 32 * k4), bd, idesc, (kc | k4) != 0);
            mma_tf32(dt, sw128_desc(alo + 32 * k4), bd, idesc, 1);
            if (P.nb == 2) mma_tf32(dt, sw128_desc(ahi + 32 * k4), sw128_desc(blo + 32 * k4), idesc, 1);
          }
          mma_commit(&empty[slot]);
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
      }
    }
  } else if (warp < 4) {
    // ---------------- hi / lo split of X, ||X||^2 ----------------
    const int tid = threadIdx.x - 64;  // 0..63
    double sq = 0.0;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; ok && u < nunits; u += gridDim.x) {
      const int64_t mt = u / P.n_ntiles;
      const bool count = P.norm_in && (u - mt * P.n_ntiles) == 0;  // each X tile once
      for (int kc = 0; kc < P.nkc; ++kc, ++g) {
        const uint32_t slot = g % P.nslot, ph = (g / P.nslot) & 1;
        if (!mbar_wait(&full[slot], ph, P.status)) {
          ok = false;
          break;
        }
        const float4* src = reinterpret_cast<const float4*>(base + (size_t)slot * slot_bytes);
        float4* dst = reinterpret_cast<float4*>(base + (size_t)slot * slot_bytes + CHUNK_BYTES);
        // ||X||^2: four FP32 partial sums of CHUNK_BYTES / 1024 squares each per chunk, folded into FP64
        // once per chunk (FP64 issues at 1/64 of the FP32 rate on this part)
        float4 part = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = tid; q < CHUNK_BYTES / 16; q += 64) {
          const float4 x = src[q];
          float4 l;
          l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
          l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
          l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
          l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
          dst[q] = l;
          part.x = fmaf(x.x, x.x, part.x);
          part.y = fmaf(x.y, x.y, part.y);
          part.z = fmaf(x.z, x.z, part.z);
          part.w = fmaf(x.w, x.w, part.w);
        }
        if (count) sq += ((double)part.x + (double)part.y) + ((double)part.z + (double)part.w);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[slot]);
      }
    }
    if (P.norm_in) {
      sq = warp_sum_d(sq);
      if (lane == 0) atomicAdd(P.norm_in, sq);
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp - 4;  // TMEM lane quarter
    double sq = 0.0, rq = 0.0;
    uint32_t it = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x, ++it) {
      const int64_t mt = u / P.n_ntiles;
      const int nt = (int)(u - mt * P.n_ntiles);
      const uint32_t acc = it & 1, aph = (it >> 1) & 1;
      if (!mbar_wait(&tfull[acc], aph, P.status)) break;
      fence_after();
      const int64_t row = mt * BM + q * 32 + lane;
      const bool valid = row < P.rows;
      int64_t o = 0, i = 0;
      if (valid) {
        o = row / P.R2;
        i = row - o * P.R2;
      }
      const int s0 = nt * P.S_tile;
      float* dst = P.out + (o * P.S_store) * P.R2 + i;
      for (int c0 = 0; c0 < P.S_tile && s0 + c0 < P.S; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + acc * P.S_tile + c0, v);
        if (valid) {
          float part = 0.f, rpart = 0.f;  // 16 squares in FP32, folded into FP64 once
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int s = s0 + c0 + j;
            if (s < P.S_store) {
              dst[(int64_t)s * P.R2] = v[j];
              part = fmaf(v[j], v[j], part);
            } else if (s < P.S) {
              rpart = fmaf(v[j], v[j], rpart);
            }
          }
          if (P.norm_out) sq += (double)part;
          if (P.resid) rq += (double)rpart;
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
    if (P.norm_out) {
      sq = warp_sum_d(sq);
      if (lane == 0) atomicAdd(P.norm_out, sq);
    }
    if (P.resid) {
      rq = warp_sum_d(rq);
      if (lane == 0) atomicAdd(P.resid, rq);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// W[b][s][k] (b = 0: RN-rounded TF32 of M; b = 1: RN-rounded TF32 of the remainder), zero padded,
// with M(s, k) from U for s < S1 and from U2 for S1 <= s < S1 + S2; rows k >= Kv (the padding of a
// zero-padded input axis) are zero.
__global__ void prep_weights_kernel(const double* __restrict__ U, const double* __restrict__ U2, int64_t Kv,
                                    int64_t S1, int64_t S2, int64_t ldu, int64_t ldu2, int transpose,
                                    float* __restrict__ W, int S_pad, int K_pad, int nb) {
  const int64_t total = (int64_t)S_pad * K_pad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / K_pad, k = e - s * K_pad;
    float x = 0.f;
    if (k < Kv) {
      if (s < S1)
        x = (float)(transpose ? U[k * ldu + s] : U[s * ldu + k]);
      else if (s < S1 + S2)
        x = (float)(transpose ? U2[k * ldu2 + (s - S1)] : U2[(s - S1) * ldu2 + k]);
    }
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    const float xh = __uint_as_float(h);
    W[e] = xh;
    if (nb == 2) {
      uint32_t l;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - xh));
      W[total + e] = __uint_as_float(l);
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map_2d(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint32_t box_inner,
                 uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * 4};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

bool ttm_tc_supported(int64_t K, int64_t S, int nb) {
  return K >= 4 && K % 4 == 0 && S >= 1 && S <= 4096 && nb >= 1 && nb <= 2;
}

size_t ttm_tc_weights_bytes(int64_t K, int64_t S) {
  const int64_t S_pad = (S + 15) / 16 * 16, K_pad = (K + 31) / 32 * 32;
  return (size_t)2 * S_pad * K_pad * sizeof(float);
}

cudaError_t launch_prep_tc_weights(const double* U, int64_t K, int64_t S, int64_t ldu, bool transpose, float* W,
                                   int nb, cudaStream_t s) {
  return launch_prep_tc_weights2(U, S, ldu, nullptr, 0, 1, K, transpose, W, nb, s);
}

cudaError_t launch_prep_tc_weights2(const double* U, int64_t S1, int64_t ldu, const double* U2, int64_t S2,
                                    int64_t ldu2, int64_t K, bool transpose, float* W, int nb, cudaStream_t s,
                                    int64_t k_valid) {
  const int64_t S = S1 + S2;
  const int S_pad = (int)((S + 15) / 16 * 16), K_pad = (int)((K + 31) / 32 * 32);
  const int64_t Kv = (k_valid < 0) ? K : std::min(k_valid, K);
  ProfScope prof(K_COPY, s);
  prep_weights_kernel<<<64, 256, 0, s>>>(U, U2, Kv, S1, S2, ldu, ldu2, transpose ? 1 : 0, W, S_pad, K_pad, nb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ttm_tc(const float* X, int64_t rows, int64_t K, const float* W, int64_t S, int nb, float* out,
                          int64_t R2, double* norm_in, double* norm_out, int* status, cudaStream_t s) {
  return launch_ttm_tc_resid(X, rows, K, W, S, S, nb, out, R2, norm_in, norm_out, nullptr, status, s);
}

cudaError_t launch_ttm_tc_resid(const float* X, int64_t rows, int64_t K, const float* W, int64_t S, int64_t S_store,
                                int nb, float* out, int64_t R2, double* norm_in, double* norm_out, double* resid,
                                int* status, cudaStream_t s) {
  if (!ttm_tc_supported(K, S, nb) || rows <= 0 || R2 <= 0 || S_store < 0 || S_store > S) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0 || (reinterpret_cast<uintptr_t>(W) & 15) != 0)
    return cudaErrorInvalidValue;
  const int S_pad = (int)((S + 15) / 16 * 16), K_pad = (int)((K + 31) / 32 * 32);
  // MMA N per unit: the whole padded output when it fits (<= 256), else balanced tiles of <= 256
  const int n_ntiles = (S_pad + 255) / 256;
  const int S_tile = ((S_pad + n_ntiles - 1) / n_ntiles + 15) / 16 * 16;
  const int nkc = K_pad / KC;
  const int w_bytes = S_tile * 128;
  const int slot_bytes = 2 * CHUNK_BYTES + nb * w_bytes;
  const int nslot = std::max(2, std::min(6, (200 * 1024) / slot_bytes));
  CUtensorMap mx, mw;
  if (!make_map_2d(&mx, X, (uint64_t)K, (uint64_t)rows, KC, BM)) return cudaErrorInvalidValue;
  if (!make_map_2d(&mw, W, (uint64_t)K_pad, (uint64_t)S_pad * nb, KC, (uint32_t)S_tile)) return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)nslot * slot_bytes + (size_t)(3 * nslot + 4) * 8;
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(ttm_tc_kernel));
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nunits = ((rows + BM - 1) / BM) * n_ntiles;
  const int grid = (int)std::min<int64_t>(nunits, nsm);
  TcParams P{rows, nkc, (int)S, (int)S_store, S_pad, S_tile, n_ntiles, nb, nslot, R2, out, norm_in, norm_out, resid,
             status};
  ProfScope prof(K_TTM_TC, s, 2.0 * (double)rows * (double)K * (double)S,
                 4.0 * (double)rows * ((double)K + (double)S_store));
  ttm_tc_kernel<<<grid, TC_THREADS, smem, s>>>(mx, mw, P);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

// pair.cu — single-read passes over two adjacent modes (a, b) of a layer intermediate viewed as
// X[A][na][nb][B] (B contiguous, fp32), for the small leaves of a dimension tree:
//
//   pair_gram    : G_a = X_(a) X_(a)^T and G_b = X_(b) X_(b)^T, the Gram matrices of both mode
//                  unfoldings (the error-truncated SVD of eq. ht_leaf_svd is taken through them), in
//                  one read of X;
//   pair_project : out[A][ra][rb][B] = X x_a U_a^T x_b U_b^T (eq. ht_leaf_contraction for both modes,
//                  and Step 1 of Algorithm 2), with ||X||^2 and ||out||^2.
//
// These passes are HBM-bound (a few to twenty-five FMAs per element for leaves of at most 24 or 32
// rows), so they run on the FP32 SIMT pipes; a tile is the full (na, nb) block for 32 consecutive
// columns of B, staged by 3-D TMA loads with the 128-byte swizzle (conflict-free column reads) in a
// ring of shared-memory stages (two whole tiles for the Gram pass, up to six half-tile bands for the
// projection), by persistent CTAs (one per SM). Lanes of a warp own the 32 columns of a tile.
//
// Precision: products and sums in FP32 with round-to-nearest (no bias in any sum of squares); the Gram
// pass keeps FP32 partial sums per lane and folds them into FP64 every few tiles, the projection folds
// per-tile FP32 norms into FP64. Every TMA wait is bounded; a wait that gives up sets the status word
// (BHT_ETIMEOUT), the CTA drains its loads in flight (again bounded) and returns.
#include <algorithm>

#include "bht.h"
#include "internal.cuh"
#include "tcgen.cuh"
#include "tma.cuh"

namespace bht {
namespace {

constexpr int PCOLS = 32;               // columns of B per tile (one swizzled 128-byte row)
constexpr int PAIR_MAX_GRAM = 24;       // mode sizes of the Gram pass (8 x 8 blocks, <= 12 warps)
constexpr int PAIR_MAX_PROJ = 32;       // mode sizes of the projection pass
constexpr int PROJ_THREADS = 384;
constexpr int GRAM_FOLD = 8;            // tiles between FP64 folds of the Gram partial sums
constexpr uint64_t DRAIN_NS = 100000000ull;

struct PairGeom {
  int64_t A, B, ncb, ntiles;
  int na, nb;
  uint32_t tile_bytes;   // na * nb * 128
  uint32_t stage_bytes;  // tile_bytes rounded up to 1024
};

__device__ __forceinline__ float tile_at(const uint8_t* T, uint32_t row, uint32_t c) {
  return *reinterpret_cast<const float*>(T + tma::sw128_offset(row, c));
}

__device__ __forceinline__ void issue_tile(const CUtensorMap* map, uint64_t* bar, uint8_t* buf, const PairGeom& g,
                                           int64_t t) {
  const int64_t a = t / g.ncb, cb = t - a * g.ncb;
  tma::mbar_expect_tx(bar, g.tile_bytes);
  tma::load_3d(map, bar, buf, (int)(cb * PCOLS), 0, (int)(a * g.na));
}

// After a failed wait: wait (bounded, ignoring the status word) for the loads this CTA still has in
// flight, so that no copy lands in shared memory after the CTA has left.
__device__ void drain_loads(uint64_t* full, const int64_t* issued, int64_t done0, int64_t done1) {
  const int64_t done[2] = {done0, done1};
  for (int s = 0; s < 2; ++s) {
    for (int64_t n = done[s]; n < issued[s]; ++n) {
      const uint32_t par = (uint32_t)(n & 1);
      const uint64_t t0 = tma::gtimer();
      uint32_t ok = 0;
      while (!ok && tma::gtimer() - t0 < DRAIN_NS) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tma::smem_u32(&full[s])), "r"(par)
            : "memory");
      }
      if (!ok) return;
    }
  }
}

__device__ __forceinline__ double block_sum2(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < nw) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid on thread 0
}

// ---------------------------------------------------------------------------------------------
// Projection of both modes. The unit of work is a band of ka rows of mode a (ka = ceil(na / 2) for
// na >= 16, else na) of one tile, staged NST units deep. Stage 1: Z[i][b][c] = sum_j T[i][j][c] Ub[j][b]
// (one thread per (i, c)). Stage 2: W[a][b][c] += sum_i Ua[i][a] Z[i][b][c] (one thread per (b, c),
// accumulated in registers over the bands of a tile), stored after the last band with the 32 lanes of
// a warp on 32 consecutive columns.
// ---------------------------------------------------------------------------------------------
constexpr int PROJ_STAGES_MAX = 6;

struct ProjGeom {
  int ka, nbands, nst;
  uint32_t unit_bytes, stage_bytes;
};

__device__ __forceinline__ void issue_band(const CUtensorMap* map, uint64_t* bar, uint8_t* buf, const PairGeom& g,
                                           const ProjGeom& pg, int64_t u) {
  const int64_t t = u / pg.nbands;
  const int band = (int)(u - t * pg.nbands);
  const int64_t a = t / g.ncb, cb = t - a * g.ncb;
  tma::mbar_expect_tx(bar, pg.unit_bytes);
  tma::load_3d(map, bar, buf, (int)(cb * PCOLS), 0, (int)(a * g.na + band * pg.ka));
}

// The next band a CTA loads, advanced without divisions: (item row block a, column block cb, band).
struct BandCursor {
  int a, cb, band;
  __device__ void start(int64_t tile, const PairGeom& g) {
    a = (int)(tile / g.ncb);
    cb = (int)(tile - (int64_t)a * g.ncb);
    band = 0;
  }
  __device__ __forceinline__ void issue(const CUtensorMap* map, uint64_t* bar, uint8_t* buf, const PairGeom& g,
                                        const ProjGeom& pg) {
    tma::mbar_expect_tx(bar, pg.unit_bytes);
    tma::load_3d(map, bar, buf, cb * PCOLS, 0, a * g.na + band * pg.ka);
    if (++band == pg.nbands) {
      band = 0;
      if (++cb == (int)g.ncb) {
        cb = 0;
        ++a;
      }
    }
  }
};

template <int RA, int RB>
__global__ void __launch_bounds__(PROJ_THREADS, 1)
    pair_project_kernel(const __grid_constant__ CUtensorMap map, const PairGeom g, const ProjGeom pg,
                        const double* __restrict__ Ua, int ra, int lda, const double* __restrict__ Ub, int rb,
                        int ldb, float* __restrict__ out, double* norm_in, double* norm_out, double* resid,
                        int* status) {
  extern __shared__ __align__(1024) uint8_t psm[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(psm) + 1023) & ~(uintptr_t)1023);
  float* Z = reinterpret_cast<float*>(base + (size_t)pg.nst * pg.stage_bytes);  // [ka][RB][32]
  float* Uas = Z + (size_t)pg.ka * RB * PCOLS;                                   // [na][RA]
  float* Ubs = Uas + (size_t)g.na * RA;                                          // [nb][RB]
  __shared__ __align__(8) uint64_t full[PROJ_STAGES_MAX];
  __shared__ double red[32];
  const int tid = threadIdx.x;
  for (int e = tid; e < g.na * RA; e += blockDim.x) {
    const int i = e / RA, a = e - i * RA;
    Uas[e] = a < ra ? (float)Ua[(int64_t)i * lda + a] : 0.f;
  }
  for (int e = tid; e < g.nb * RB; e += blockDim.x) {
    const int j = e / RB, b = e - j * RB;
    Ubs[e] = b < rb ? (float)Ub[(int64_t)j * ldb + b] : 0.f;
  }
  if (tid == 0) {
    for (int s = 0; s < pg.nst; ++s) tma::mbar_init(&full[s], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  // this CTA's units: the bands of its tiles t = blockIdx.x + k * gridDim.x, in order
  const int64_t G = gridDim.x;
  const int64_t my_tiles = (g.ntiles > blockIdx.x) ? (g.ntiles - 1 - blockIdx.x) / G + 1 : 0;
  const int64_t my_units = my_tiles * pg.nbands;
  auto unit_id = [&](int64_t k) { return (blockIdx.x + (k / pg.nbands) * G) * pg.nbands + k % pg.nbands; };
  int64_t issued = 0;
  if (tid == 0)
    for (; issued < my_units && issued < pg.nst; ++issued)
      issue_band(&map, &full[issued], base + (size_t)issued * pg.stage_bytes, g, pg, unit_id(issued));
  double sx = 0.0, sy = 0.0;
  float acc2[2][RA];  // stage 2: the pairs q = tid and q = tid + PROJ_THREADS
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int a = 0; a < RA; ++a) acc2[h][a] = 0.f;
  for (int64_t k = 0; k < my_units; ++k) {
    const int s = (int)(k % pg.nst);
    const bool got = tma::mbar_wait(&full[s], (uint32_t)((k / pg.nst) & 1), status);
    if (!__syncthreads_and(got)) {
      if (tid == 0) {
        // drain: the loads of units k .. issued-1 are in flight, one per stage
        for (int64_t q = k; q < issued; ++q) {
          const uint64_t t0 = tma::gtimer();
          uint32_t ok = 0;
          const int sq = (int)(q % pg.nst);
          while (!ok && tma::gtimer() - t0 < DRAIN_NS) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(tma::smem_u32(&full[sq])), "r"((uint32_t)((q / pg.nst) & 1))
                : "memory");
          }
          if (!ok) break;
        }
      }
      break;
    }
    const int band = (int)(k % pg.nbands);
    const int64_t t = blockIdx.x + (k / pg.nbands) * G;
    const uint8_t* T = base + (size_t)s * pg.stage_bytes;
    const int i0 = band * pg.ka;
    const int kv = min(pg.ka, g.na - i0);  // rows of this band inside mode a
    float xx = 0.f;
    for (int p = tid; p < kv * PCOLS; p += blockDim.x) {
      const int i = p >> 5, c = p & 31;
      float acc[RB];
#pragma unroll
      for (int b = 0; b < RB; ++b) acc[b] = 0.f;
      // rows r = i nb + j: the swizzle depends on r mod 8 only, so eight base addresses serve every j
      const uint32_t r0 = (uint32_t)(i * g.nb);
      const uint8_t* rb8[8];
#pragma unroll
      for (int k8 = 0; k8 < 8; ++k8) rb8[k8] = T + tma::sw128_offset(r0 + k8, (uint32_t)c);
      int j = 0;
      for (; j + 8 <= g.nb; j += 8) {
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
          const float x = *reinterpret_cast<const float*>(rb8[k8] + (size_t)j * 128);
          xx = fmaf(x, x, xx);
          const float4* u = reinterpret_cast<const float4*>(Ubs + (j + k8) * RB);
#pragma unroll
          for (int b4 = 0; b4 < RB / 4; ++b4) {
            const float4 w = u[b4];
            acc[4 * b4 + 0] = fmaf(x, w.x, acc[4 * b4 + 0]);
            acc[4 * b4 + 1] = fmaf(x, w.y, acc[4 * b4 + 1]);
            acc[4 * b4 + 2] = fmaf(x, w.z, acc[4 * b4 + 2]);
            acc[4 * b4 + 3] = fmaf(x, w.w, acc[4 * b4 + 3]);
          }
        }
      }
      for (; j < g.nb; ++j) {
        const float x = tile_at(T, r0 + (uint32_t)j, (uint32_t)c);
        xx = fmaf(x, x, xx);
        const float4* u = reinterpret_cast<const float4*>(Ubs + j * RB);
#pragma unroll
        for (int b4 = 0; b4 < RB / 4; ++b4) {
          const float4 w = u[b4];
          acc[4 * b4 + 0] = fmaf(x, w.x, acc[4 * b4 + 0]);
          acc[4 * b4 + 1] = fmaf(x, w.y, acc[4 * b4 + 1]);
          acc[4 * b4 + 2] = fmaf(x, w.z, acc[4 * b4 + 2]);
          acc[4 * b4 + 3] = fmaf(x, w.w, acc[4 * b4 + 3]);
        }
      }
#pragma unroll
      for (int b = 0; b < RB; ++b) Z[(i * RB + b) * PCOLS + c] = acc[b];
    }
    sx += (double)xx;
    __syncthreads();  // Z complete; every read of this stage done
    if (tid == 0 && issued < my_units) {
      issue_band(&map, &full[issued % pg.nst], base + (size_t)(issued % pg.nst) * pg.stage_bytes, g, pg,
                 unit_id(issued));
      ++issued;
    }
    float yy = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + h * PROJ_THREADS;
      if (q >= rb * PCOLS) break;
      const int b = q >> 5, c = q & 31;
#pragma unroll 4
      for (int i = 0; i < kv; ++i) {
        const float z = Z[(i * RB + b) * PCOLS + c];
        const float4* u = reinterpret_cast<const float4*>(Uas + (i0 + i) * RA);
#pragma unroll
        for (int a4 = 0; a4 < RA / 4; ++a4) {
          const float4 w = u[a4];
          acc2[h][4 * a4 + 0] = fmaf(z, w.x, acc2[h][4 * a4 + 0]);
          acc2[h][4 * a4 + 1] = fmaf(z, w.y, acc2[h][4 * a4 + 1]);
          acc2[h][4 * a4 + 2] = fmaf(z, w.z, acc2[h][4 * a4 + 2]);
          acc2[h][4 * a4 + 3] = fmaf(z, w.w, acc2[h][4 * a4 + 3]);
        }
      }
      if (band == pg.nbands - 1) {
        const int64_t aidx = t / g.ncb, col = (t - aidx * g.ncb) * PCOLS + c;
        if (col < g.B) {
          float* o = out + ((aidx * ra) * rb + b) * g.B + col;
#pragma unroll
          for (int a = 0; a < RA; ++a)
            if (a < ra) {
              o[(int64_t)a * rb * g.B] = acc2[h][a];
              yy = fmaf(acc2[h][a], acc2[h][a], yy);
            }
        }
#pragma unroll
        for (int a = 0; a < RA; ++a) acc2[h][a] = 0.f;
      }
    }
    sy += (double)yy;
    __syncthreads();  // Z consumed before the next band's stage 1
  }
  sx = block_sum2(sx, red);
  sy = block_sum2(sy, red);
  if (tid == 0) {
    if (norm_in) atomicAdd(norm_in, sx);
    if (norm_out) atomicAdd(norm_out, sy);
    if (resid) atomicAdd(resid, sx - sy);
  }
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised projection for ranks <= 8, na = nb = 24. The basis entries a lane needs live in
// its registers, so no basis is ever re-read from shared memory.
//   stage 1 (ka warps, warp i = row i of a band of ka rows): Z[i][b][c] = sum_j T[i][j][c] Ub[j][b].
//   Lane (g, p) = lane (8 p + g) owns the four columns 4g .. 4g+3 and the six rows j = p, p+4, ...;
//   a quarter-warp reads one whole 128-byte row, so every 16-byte load is a distinct word of shared
//   memory and feeds 32 FMAs (all eight outputs b). The four partial sums of an output are then
//   reduce-scattered over the lanes p = 0..3 with two rounds of shuffles, after which lane p holds
//   outputs p and p + 4. Lane p keeps its outputs in the order b = slot XOR p (its basis registers
//   are loaded in that order), so both rounds keep the even / low slots without any select.
//   stage 2 (4 warps, warp w: b = w and w + 4): W[a][b][c] = sum_i Ua[i][a] Z[i][b][c] over the na
//   rows of a tile; lane (g, p) owns the four columns 4g .. 4g+3 and a = p, p + 4; once per tile,
//   written with 16-byte stores.
// A unit is one band of ka rows of mode a; two bands make a tile. Z holds one band and is
// triple-buffered by unit index, handed over through named barriers:
//   ZFULL[z] (ids 2, 3, 4): stage 1 arrives after it has written Z[z] (and read the band's TMA
//   stage), stage 2 waits; ZEMPTY[z] (ids 5, 6, 7): stage 2 arrives when it has read Z[z], stage 1
//   waits before it writes Z[z] again; S1 (id 1): the stage-1 warps among themselves.
// Thread 0 alone waits on each TMA barrier (bounded) and tells the stage-1 warps through shared memory;
// the first stage-2 thread issues the loads, refilling a stage once ZFULL says stage 1 is done with
// it, and walks the bands with a cursor (no integer division on the way). A wait that gave up raises
// an abort flag that stage 2 reads after its next ZFULL wait, so every named barrier still sees
// matching arrivals on both sides and both roles leave together.
// ---------------------------------------------------------------------------------------------
constexpr int WS_W2 = 4;  // stage-2 warps, two output indices of mode b each
constexpr int WS_MAX_THREADS = 32 * (12 + WS_W2);

// Knuth's TwoSum into a double-single accumulator (hi, lo): sums of norms kept in FP32 at FP64-class
// accuracy (the FP64 pipes of this part issue at 1/64 of the FP32 rate).
__device__ __forceinline__ void ds_add(float v, float& hi, float& lo) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

// Packed FP32 FMA on register pairs (two independent round-to-nearest FMAs).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int NB, int KA>
__global__ void __launch_bounds__(WS_MAX_THREADS, 1)
    pair_project_ws_kernel(const __grid_constant__ CUtensorMap map, const PairGeom g, const ProjGeom pg,
                           const double* __restrict__ Ua, int ra, int lda, const double* __restrict__ Ub, int rb,
                           int ldb, float* __restrict__ out, double* norm_in, double* norm_out, double* resid,
                           int* status) {
  constexpr int NA = 2 * KA;  // rows of mode a held in stage 2's registers: two bands of KA rows
  constexpr int NZ = 3;       // Z buffers
  extern __shared__ __align__(1024) uint8_t wsm[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(wsm) + 1023) & ~(uintptr_t)1023);
  float* Zb = reinterpret_cast<float*>(base + (size_t)pg.nst * pg.stage_bytes);  // [NZ][KA][8][32]
  __shared__ __align__(8) uint64_t full[PROJ_STAGES_MAX];
  __shared__ int sflag[2], abort_flag;
  __shared__ double red[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int W1 = pg.ka, NT = (int)blockDim.x;
  const int gq = lane >> 2, pq = lane & 3;  // stage 2: columns 4 gq .. 4 gq + 3, outputs a = pq, pq + 4
  const size_t zsize = (size_t)KA * 8 * PCOLS;
  if (tid == 0) {
    for (int st = 0; st < pg.nst; ++st) tma::mbar_init(&full[st], 1);
    tma::fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  // each CTA takes a contiguous run of tiles (consecutive column blocks of the same rows), so that its
  // successive loads continue the DRAM pages of its previous ones
  // (the launcher keeps ntiles * nbands below 2^31, so tile and unit counters fit 32 bits)
  const int per = (int)((g.ntiles + gridDim.x - 1) / gridDim.x);
  const int t0 = (int)blockIdx.x * per;
  const int my_tiles = (g.ntiles > t0) ? min(per, (int)g.ntiles - t0) : 0;
  const int my_units = my_tiles * pg.nbands;
  double sx = 0.0, sy = 0.0;
  if (warp < W1) {
    // ---------------- stage 1 ----------------
    static_assert(NB % 8 == 0, "rows of a warp start on a swizzle period");
    constexpr int JR = NB / 4;              // rows j = 4 m + p of lane (g, p), m < JR
    const int g1 = lane & 7, p1 = lane >> 3;  // stage-1 lane (g1, p1)
    float2 u[JR][4];  // u[m][h] = (Ub[4 m + p1][2h ^ p1], Ub[4 m + p1][(2h + 1) ^ p1]): slots 2h, 2h + 1
#pragma unroll
    for (int m = 0; m < JR; ++m)
#pragma unroll
      for (int hh = 0; hh < 4; ++hh) {
        const int j = 4 * m + p1, b0 = (2 * hh) ^ p1, b1 = (2 * hh + 1) ^ p1;
        u[m][hh].x = (j < g.nb && b0 < rb) ? (float)Ub[(int64_t)j * ldb + b0] : 0.f;
        u[m][hh].y = (j < g.nb && b1 < rb) ? (float)Ub[(int64_t)j * ldb + b1] : 0.f;
      }
    int k = 0, posted = 0;  // units consumed; Z buffers handed to stage 2
    int s = 0, zb = 0;
    float sx_hi = 0.f, sx_lo = 0.f;
    uint32_t par = 0;
    for (; k < my_units; ++k) {
      // the verdict of the wait is double-buffered: thread 0 may run one unit ahead of a slow warp
      if (tid == 0) sflag[k & 1] = tma::mbar_wait(&full[s], par, status) ? 0 : 1;
      named_sync(1, 32 * W1);
      const bool abort_now = sflag[k & 1] != 0;
      if (k >= NZ) named_sync(5 + zb, NT);  // stage 2 has read Z[zb] (unit k - NZ)
      if (abort_now) {
        if (tid == 0) abort_flag = 1;
        named_arrive(2 + zb, NT);  // wake stage 2 for unit k; it sees the flag and leaves
        ++posted;
        break;
      }
      const uint8_t* T = base + (size_t)s * pg.stage_bytes;
      if (warp < KA) {
        float2 acc[4][4];  // acc[c][h] = slots (2h, 2h + 1) of column c, two FMAs per packed instruction
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int hh = 0; hh < 4; ++hh) acc[c][hh] = make_float2(0.f, 0.f);
        float2 xx2 = make_float2(0.f, 0.f);
        // row r = warp NB + 4 m + p1 has swizzle (4 m + p1) mod 8 = 4 (m mod 2) + p1, so the 16-byte
        // chunk of columns 4 g1 .. 4 g1 + 3 sits at g1 ^ p1 ^ 4 (m mod 2)
        const uint8_t* Tw = T + (size_t)(warp * NB + p1) * 128;
        const int ch = g1 ^ p1;
#pragma unroll
        for (int m = 0; m < JR; ++m) {
          const float4 x = *reinterpret_cast<const float4*>(Tw + m * 512 + ((ch ^ ((m & 1) << 2)) << 4));
          xx2 = ffma2(make_float2(x.x, x.y), make_float2(x.x, x.y), xx2);
          xx2 = ffma2(make_float2(x.z, x.w), make_float2(x.z, x.w), xx2);
          const float xc[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float2 xd = make_float2(xc[c], xc[c]);
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) acc[c][hh] = ffma2(xd, u[m][hh], acc[c][hh]);
          }
        }
        // reduce-scatter over p1: the partner p1 ^ 1 holds in slot 2h + 1 the output that slot 2h
        // holds here, and p1 ^ 2 in slot 4h' + 2 what slot 4h' holds here
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int hh = 0; hh < 4; ++hh) acc[c][hh].x += __shfl_xor_sync(0xffffffffu, acc[c][hh].y, 8);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c][0].x += __shfl_xor_sync(0xffffffffu, acc[c][1].x, 16);
          acc[c][2].x += __shfl_xor_sync(0xffffffffu, acc[c][3].x, 16);
        }
        // slots 0 and 4 hold outputs p1 and p1 + 4
        float* Z = Zb + (size_t)zb * zsize + (size_t)(warp * 8 + p1) * PCOLS + 4 * g1;
        *reinterpret_cast<float4*>(Z) = make_float4(acc[0][0].x, acc[1][0].x, acc[2][0].x, acc[3][0].x);
        *reinterpret_cast<float4*>(Z + 4 * PCOLS) = make_float4(acc[0][2].x, acc[1][2].x, acc[2][2].x, acc[3][2].x);
        ds_add(xx2.x + xx2.y, sx_hi, sx_lo);
      }
      if (++s == pg.nst) {
        s = 0;
        par ^= 1u;
      }
      // Z[zb] holds this band, and every stage-1 read of this band's stage is done: stage 2 refills it
      named_arrive(2 + zb, NT);
      ++posted;
      if (++zb == NZ) zb = 0;
    }
    // the Z buffers of the last (up to) NZ units posted: wait until stage 2 has read them
    for (int q = (posted >= NZ ? posted - NZ : 0); q < posted; ++q) named_sync(5 + q % NZ, NT);
    // every element of a band was squared by exactly one lane
    sx = (double)sx_hi + (double)sx_lo;
  } else {
    // ---------------- stage 2 ----------------
    const int b0 = warp - W1, b1 = b0 + WS_W2;  // output indices of mode b of this warp
    float4 v[NA];  // (Ua[i][pq], Ua[i][pq], Ua[i][pq + 4], Ua[i][pq + 4]): each basis entry twice, so a
                   // packed FMA takes two columns of Z against it without any register copy
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const float x0 = (i < g.na && pq < ra) ? (float)Ua[(int64_t)i * lda + pq] : 0.f;
      const float x1 = (i < g.na && pq + 4 < ra) ? (float)Ua[(int64_t)i * lda + pq + 4] : 0.f;
      v[i] = make_float4(x0, x0, x1, x1);
    }
    float2 acc[2][2][2];  // acc[b0 or b1][a = pq or pq + 4][columns (0, 1) or (2, 3)]
#pragma unroll
    for (int hb = 0; hb < 2; ++hb)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) acc[hb][h][cp] = make_float2(0.f, 0.f);
    float sy_hi = 0.f, sy_lo = 0.f;
    // the first stage-2 thread issues the TMA loads: unit u goes to stage u mod nst, refilled once
    // stage 1 has posted the band that occupied it
    const bool producer = tid == 32 * W1;
    int issued = 0, sq = 0;  // units issued; the stage of the next one
    BandCursor cur;
    if (producer) {
      cur.start(t0, g);
      for (; issued < my_units && issued < pg.nst; ++issued)
        cur.issue(&map, &full[issued], base + (size_t)issued * pg.stage_bytes, g, pg);
    }
    // the item row block and column block of the tile being accumulated
    int oa = (int)(t0 / g.ncb), ocb = (int)(t0 - (int64_t)oa * g.ncb);
    int k = 0, zb = 0;
    for (; k < my_units; ++k) {
      const int band = k & 1;  // two bands per tile
      named_sync(2 + zb, NT);
      if (abort_flag) {
        named_arrive(5 + zb, NT);
        break;
      }
      if (producer && issued < my_units) {
        // sq == issued mod nst == k mod nst: the stage unit k has just left
        cur.issue(&map, &full[sq], base + (size_t)sq * pg.stage_bytes, g, pg);
        ++issued;
        if (++sq == pg.nst) sq = 0;
      }
      const float* Z = Zb + (size_t)zb * zsize + 4 * gq;
      // one unrolled copy per band, so the basis rows are picked at compile time
      auto rows = [&](const float4* vb) {
#pragma unroll
        for (int i = 0; i < KA; ++i) {
          const float4 za = *reinterpret_cast<const float4*>(Z + (size_t)(i * 8 + b0) * PCOLS);
          const float4 zc = *reinterpret_cast<const float4*>(Z + (size_t)(i * 8 + b1) * PCOLS);
          const float2 w0 = make_float2(vb[i].x, vb[i].y), w1 = make_float2(vb[i].z, vb[i].w);
          acc[0][0][0] = ffma2(make_float2(za.x, za.y), w0, acc[0][0][0]);
          acc[0][0][1] = ffma2(make_float2(za.z, za.w), w0, acc[0][0][1]);
          acc[0][1][0] = ffma2(make_float2(za.x, za.y), w1, acc[0][1][0]);
          acc[0][1][1] = ffma2(make_float2(za.z, za.w), w1, acc[0][1][1]);
          acc[1][0][0] = ffma2(make_float2(zc.x, zc.y), w0, acc[1][0][0]);
          acc[1][0][1] = ffma2(make_float2(zc.z, zc.w), w0, acc[1][0][1]);
          acc[1][1][0] = ffma2(make_float2(zc.x, zc.y), w1, acc[1][1][0]);
          acc[1][1][1] = ffma2(make_float2(zc.z, zc.w), w1, acc[1][1][1]);
        }
      };
      if (band)
        rows(v + KA);
      else
        rows(v);
      named_arrive(5 + zb, NT);  // Z[zb] read
      if (++zb == NZ) zb = 0;
      if (band == 1) {
        const int64_t aidx = oa;
        const int col = ocb * PCOLS + 4 * gq;
        if (col < g.B) {  // B % 4 == 0, so the four columns are all inside
          float yy = 0.f;
#pragma unroll
          for (int hb = 0; hb < 2; ++hb) {
            const int b = hb ? b1 : b0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int a = pq + 4 * h;
              if (b < rb && a < ra) {
                const float4 w = make_float4(acc[hb][h][0].x, acc[hb][h][0].y, acc[hb][h][1].x, acc[hb][h][1].y);
                *reinterpret_cast<float4*>(out + ((aidx * ra + a) * rb + b) * g.B + col) = w;
                yy = fmaf(w.x, w.x, fmaf(w.y, w.y, fmaf(w.z, w.z, fmaf(w.w, w.w, yy))));
              }
            }
          }
          ds_add(yy, sy_hi, sy_lo);
        }
#pragma unroll
        for (int hb = 0; hb < 2; ++hb)
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int cp = 0; cp < 2; ++cp) acc[hb][h][cp] = make_float2(0.f, 0.f);
        if (++ocb == (int)g.ncb) {
          ocb = 0;
          ++oa;
        }
      }
    }
    if (producer && k < my_units) {
      // stage 1 gave up on a wait: drain the loads still in flight (bounded, ignoring the status word)
      for (int q = k; q < issued; ++q) {
        const int sq = q % pg.nst;
        const uint32_t pp = (uint32_t)((q / pg.nst) & 1);
        const uint64_t tw = tma::gtimer();
        uint32_t ok = 0;
        while (!ok && tma::gtimer() - tw < DRAIN_NS) {
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(ok)
              : "r"(tma::smem_u32(&full[sq])), "r"(pp)
              : "memory");
        }
        if (!ok) break;
      }
    }
    sy = (double)sy_hi + (double)sy_lo;
  }
  __syncthreads();
  sx = block_sum2(sx, red);
  sy = block_sum2(sy, red);
  if (tid == 0) {
    if (norm_in) atomicAdd(norm_in, sx);
    if (norm_out) atomicAdd(norm_out, sy);
    if (resid) atomicAdd(resid, sx - sy);
  }
}

// ---------------------------------------------------------------------------------------------
// Gram matrices of both modes. Warp w owns one 8 x 8 block (p <= q) of the upper triangle of G_a
// (warps 0 .. wa-1) or of G_b (the rest); lane c accumulates its column's outer products in FP32,
// G_a over (j, c) and G_b over (i, c); every GRAM_FOLD tiles the warp sums its lanes and adds the
// block into FP64 shared memory, which is added to G (both triangles) once per CTA.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void block_of(int w, int n8, int& p, int& q) {
  int t = w;
  p = 0;
  while (t >= n8 - p) {
    t -= n8 - p;
    ++p;
  }
  q = p + t;
}

__device__ __forceinline__ void fold_block(float (&acc)[8][8], double* blk) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      float x = acc[u][v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == ((u * 8 + v) & 31)) blk[u * 8 + v] += (double)x;
      acc[u][v] = 0.f;
    }
}

__global__ void __launch_bounds__(384, 1)
    pair_gram_kernel(const __grid_constant__ CUtensorMap map, const PairGeom g, int wa, double* __restrict__ Ga,
                     double* __restrict__ Gb, int* status) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~(uintptr_t)1023);
  uint8_t* stage[2] = {base, base + g.stage_bytes};
  double* blocks = reinterpret_cast<double*>(base + 2 * (size_t)g.stage_bytes);  // [warps][64]
  __shared__ __align__(8) uint64_t full[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = (int)(blockDim.x >> 5);
  const bool on_a = warp < wa;
  const int n8 = on_a ? (g.na + 7) / 8 : (g.nb + 7) / 8;
  int p, q;
  block_of(on_a ? warp : warp - wa, n8, p, q);
  double* blk = blocks + warp * 64;
  for (int e = lane; e < 64; e += 32) blk[e] = 0.0;
  int64_t issued[2] = {0, 0};
  if (tid == 0) {
    tma::mbar_init(&full[0], 1);
    tma::mbar_init(&full[1], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  const int64_t G = gridDim.x;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      const int64_t t = blockIdx.x + s * G;
      if (t < g.ntiles) {
        issue_tile(&map, &full[s], stage[s], g, t);
        ++issued[s];
      }
    }
  }
  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  // rows of the two 8-row groups inside the mode, and how the tile row is formed from them
  const int outer = on_a ? g.nb : g.na;  // the index summed over together with the column
  const bool fast = (g.nb & 7) == 0;
  uint32_t qoff_p[8], qoff_q[8];  // G_b operands: byte offsets of rows 8p + u and 8q + u within a block of nb rows
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    qoff_p[u] = tma::sw128_offset((uint32_t)(8 * p + u), (uint32_t)lane);
    qoff_q[u] = tma::sw128_offset((uint32_t)(8 * q + u), (uint32_t)lane);
  }
  int64_t k = 0;
  int since = 0;
  for (int64_t t = blockIdx.x; t < g.ntiles; t += G, ++k) {
    const int s = (int)(k & 1);
    const bool got = tma::mbar_wait(&full[s], (uint32_t)((k >> 1) & 1), status);
    if (!__syncthreads_and(got)) {
      if (tid == 0) drain_loads(full, issued, (k + 1) >> 1, k >> 1);
      break;
    }
    const uint8_t* T = stage[s];
    if (fast) {
      // nb % 8 == 0: the swizzle of row r depends on r mod 8, which is o mod 8 for the rows of G_a's
      // operands and u for G_b's, so the addresses are precomputed bases plus a row offset
      const size_t row_b = (size_t)g.nb * 128;
      for (int o = 0; o < outer; ++o) {
        float vp[8], vq[8];
        if (on_a) {
          const uint32_t sw = (uint32_t)(o & 7);
          const uint8_t* bp = T + (size_t)o * 128 + ((((uint32_t)lane >> 2) ^ sw) << 4) + ((lane & 3) << 2);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            vp[u] = (8 * p + u < g.na) ? *reinterpret_cast<const float*>(bp + (size_t)(8 * p + u) * row_b) : 0.f;
            vq[u] = (8 * q + u < g.na) ? *reinterpret_cast<const float*>(bp + (size_t)(8 * q + u) * row_b) : 0.f;
          }
        } else {
          const uint8_t* bo = T + (size_t)o * row_b;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            vp[u] = (8 * p + u < g.nb) ? *reinterpret_cast<const float*>(bo + qoff_p[u]) : 0.f;
            vq[u] = (8 * q + u < g.nb) ? *reinterpret_cast<const float*>(bo + qoff_q[u]) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(vp[u], vq[v], acc[u][v]);
      }
    } else {
      for (int o = 0; o < outer; ++o) {
        float vp[8], vq[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r1 = 8 * p + u, r2 = 8 * q + u;
          if (on_a) {
            vp[u] = r1 < g.na ? tile_at(T, (uint32_t)(r1 * g.nb + o), (uint32_t)lane) : 0.f;
            vq[u] = r2 < g.na ? tile_at(T, (uint32_t)(r2 * g.nb + o), (uint32_t)lane) : 0.f;
          } else {
            vp[u] = r1 < g.nb ? tile_at(T, (uint32_t)(o * g.nb + r1), (uint32_t)lane) : 0.f;
            vq[u] = r2 < g.nb ? tile_at(T, (uint32_t)(o * g.nb + r2), (uint32_t)lane) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(vp[u], vq[v], acc[u][v]);
      }
    }
    __syncthreads();  // every read of this stage done
    if (tid == 0 && t + 2 * G < g.ntiles) {
      issue_tile(&map, &full[s], stage[s], g, t + 2 * G);
      ++issued[s];
    }
    if (++since == GRAM_FOLD) {
      since = 0;
      fold_block(acc, blk);
    }
  }
  fold_block(acc, blk);
  __syncwarp();
  double* Gm = on_a ? Ga : Gb;
  const int n = on_a ? g.na : g.nb;
  for (int e = lane; e < 64; e += 32) {
    const int u = e >> 3, v = e & 7;
    const int r = 8 * p + u, c = 8 * q + v;
    if (r < n && c < n) {
      atomicAdd(&Gm[(int64_t)r * n + c], blk[e]);
      if (p != q) atomicAdd(&Gm[(int64_t)c * n + r], blk[e]);
    }
  }
  (void)nwarps;
}

// ---------------------------------------------------------------------------------------------
// Gram matrices of both modes for na = nb = 24 (the Gram twin of the warp-specialised projection).
// Same warp roles as the generic kernel (warps 0-5: the upper 8 x 8 blocks of G_a, warps 6-11: those
// of G_b, lane = column), but with the mode sizes fixed at compile time every shared-memory address
// is a per-lane base plus an immediate, products go two at a time through packed FMAs, diagonal
// blocks load one operand, and the CTA walks its contiguous run of tiles with a cursor through a
// ring of three whole-tile stages: thread 0 waits on the next tile, and after the one CTA barrier of
// a tile (every warp is then done with the previous tile) refills that tile's stage.
// ---------------------------------------------------------------------------------------------
constexpr int G24_STAGES = 3;

template <bool DIAG, uint32_t ROW_STEP, uint32_t OSTEP>
__device__ __forceinline__ void g24_block(const uint8_t* Tp, const uint8_t* Tq, const uint32_t (&lo)[8],
                                          float2 (&acc)[8][4]) {
  // operand u of the block's first rows sits at Tp + u ROW_STEP + o OSTEP + (lane offset of that row's
  // swizzle), and of its second rows at Tq + ...; the outer index runs in three rounds of eight (one
  // swizzle period), each unrolled, which keeps the kernel's code within the instruction caches
#pragma unroll 1
  for (int ob = 0; ob < 24; ob += 8) {
#pragma unroll
    for (int oo = 0; oo < 8; ++oo) {
      float vp[8], vq[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t off = u * ROW_STEP + oo * OSTEP + lo[(ROW_STEP == 128u) ? u : oo];
        vp[u] = *reinterpret_cast<const float*>(Tp + off);
        vq[u] = DIAG ? vp[u] : *reinterpret_cast<const float*>(Tq + off);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float2 d = make_float2(vp[u], vp[u]);
#pragma unroll
        for (int v = 0; v < 4; ++v)  // a diagonal block needs only the pairs that reach its upper triangle
          if (!DIAG || 2 * v + 1 >= u) acc[u][v] = ffma2(d, make_float2(vq[2 * v], vq[2 * v + 1]), acc[u][v]);
      }
    }
    Tp += 8 * OSTEP;
    Tq += 8 * OSTEP;
  }
}

__device__ __forceinline__ void g24_fold(float2 (&acc)[8][4], double* blk) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float x = acc[u][v].x, y = acc[u][v].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == ((u * 8 + 2 * v) & 31)) blk[u * 8 + 2 * v] += (double)x;
      if (lane == ((u * 8 + 2 * v + 1) & 31)) blk[u * 8 + 2 * v + 1] += (double)y;
      acc[u][v] = make_float2(0.f, 0.f);
    }
}

__global__ void __launch_bounds__(384, 1)
    pair_gram24_kernel(const __grid_constant__ CUtensorMap map, const PairGeom g, double* __restrict__ Ga,
                       double* __restrict__ Gb, int* status) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gsm) + 1023) & ~(uintptr_t)1023);
  double* blocks = reinterpret_cast<double*>(base + G24_STAGES * (size_t)g.stage_bytes);  // [12][64]
  __shared__ __align__(8) uint64_t full[G24_STAGES];
  __shared__ int sflag[2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool on_a = warp < 6;
  int p, q;
  block_of(on_a ? warp : warp - 6, 3, p, q);
  double* blk = blocks + warp * 64;
  for (int e = lane; e < 64; e += 32) blk[e] = 0.0;
  // the CTA's contiguous run of tiles, walked with a cursor (the launcher keeps ntiles below 2^31)
  const int per = (int)((g.ntiles + gridDim.x - 1) / gridDim.x);
  const int t0 = (int)blockIdx.x * per;
  const int my = (g.ntiles > t0) ? min(per, (int)g.ntiles - t0) : 0;
  int issued = 0, ca = 0, ccb = 0;
  auto issue = [&](int st) {
    tma::mbar_expect_tx(&full[st], g.tile_bytes);
    tma::load_3d(&map, &full[st], base + (size_t)st * g.stage_bytes, ccb * PCOLS, 0, ca * 24);
    if (++ccb == (int)g.ncb) {
      ccb = 0;
      ++ca;
    }
  };
  if (tid == 0) {
    for (int st = 0; st < G24_STAGES; ++st) tma::mbar_init(&full[st], 1);
    tma::fence_mbar_init();
    ca = (int)(t0 / g.ncb);
    ccb = (int)(t0 - (int64_t)ca * g.ncb);
    for (; issued < my && issued < G24_STAGES; ++issued) issue(issued);
  }
  __syncthreads();
  // lane offsets within a 128-byte row under the 128-byte swizzle: chunk (lane / 4) ^ (row mod 8)
  uint32_t lo[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) lo[r] = ((((uint32_t)lane >> 2) ^ (uint32_t)r) << 4) + (((uint32_t)lane & 3u) << 2);
  // G_a: operand u of block row p is row (8p + u) nb + o, whose swizzle is o mod 8 (nb = 24):
  //   offset (8p + u) * 3072 + o * 128; G_b: row o nb + 8p + u, swizzle u: offset o * 3072 + (8p + u) * 128
  const uint32_t row_step = on_a ? 3072u : 128u, ostep = on_a ? 128u : 3072u;
  float2 acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = make_float2(0.f, 0.f);
  int k = 0, s = 0, since = 0;
  uint32_t par = 0;
  for (; k < my; ++k) {
    if (tid == 0) sflag[k & 1] = tma::mbar_wait(&full[s], par, status) ? 0 : 1;
    __syncthreads();  // tile k is in (or the wait gave up) and every warp is done with tile k - 1
    if (sflag[k & 1]) break;
    if (tid == 0 && k >= 1 && issued < my) {
      issue(issued % G24_STAGES);  // the stage tile k - 1 has left (issued == k - 1 + stages)
      ++issued;
    }
    const uint8_t* T = base + (size_t)s * g.stage_bytes;
    const uint8_t* Tp = T + (uint32_t)(8 * p) * row_step;
    const uint8_t* Tq = T + (uint32_t)(8 * q) * row_step;
    if (on_a) {
      if (p == q)
        g24_block<true, 3072u, 128u>(Tp, Tq, lo, acc);
      else
        g24_block<false, 3072u, 128u>(Tp, Tq, lo, acc);
    } else {
      if (p == q)
        g24_block<true, 128u, 3072u>(Tp, Tq, lo, acc);
      else
        g24_block<false, 128u, 3072u>(Tp, Tq, lo, acc);
    }
    if (++s == G24_STAGES) {
      s = 0;
      par ^= 1u;
    }
    if (++since == GRAM_FOLD) {
      since = 0;
      g24_fold(acc, blk);
    }
  }
  if (tid == 0 && k < my) {
    // a wait gave up: drain the loads still in flight (bounded, ignoring the status word)
    for (int qq = k; qq < issued; ++qq) {
      const int sq = qq % G24_STAGES;
      const uint32_t pp = (uint32_t)((qq / G24_STAGES) & 1);
      const uint64_t tw = tma::gtimer();
      uint32_t okd = 0;
      while (!okd && tma::gtimer() - tw < DRAIN_NS) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(okd)
            : "r"(tma::smem_u32(&full[sq])), "r"(pp)
            : "memory");
      }
      if (!okd) break;
    }
  }
  g24_fold(acc, blk);
  __syncwarp();
  double* Gm = on_a ? Ga : Gb;
  for (int e = lane; e < 64; e += 32) {
    const int u = e >> 3, v = e & 7;
    const int r = 8 * p + u, c = 8 * q + v;
    if (p == q && v < u) continue;  // a diagonal block holds its upper triangle
    atomicAdd(&Gm[r * 24 + c], blk[e]);
    if (r != c) atomicAdd(&Gm[c * 24 + r], blk[e]);
  }
}

// ---------------------------------------------------------------------------------------------
// Both Grams of a 24 x 24 pair on the tensor cores (tcgen05, split TF32, FP32 accumulation in TMEM,
// FP64 sums per CTA). A tile (24 x 24 rows of 32 columns) arrives as twelve bands of four rows of the
// contracted mode, each in its own ring slot:
//   * six bands of i (rows (i, j), the map of the projection): for each i, the 24 rows j form a K-major
//     operand (K = the 32 columns), and G_b += X_i X_i^T is one MMA per 8 columns;
//   * six bands of j through a second map that takes i before j (rows (j, i); the same bytes, mostly from
//     L2): for each j, G_a += X_j X_j^T.
// An MMA is M = 128 rows by N = 32 from the start of a 24-row group; rows and columns beyond 24 read the
// next group (ignored in the result; the ring is followed by a pad they may reach). Split TF32: the MMA
// reads x as its TF32 part h, a converter warp pair writes l = x - h beside it, and
// G = H H^T + L H^T + (L H^T)^T. Two TMEM sets take turns: while one accumulates a tile, one warp
// moves the other's D = H H^T and E = L H^T into FP64 registers as F = D + 2E (the symmetric part of
// the sum of the F is G, D being symmetric).
// Warps: 0 TMA producer, 1 TMEM allocation and MMA issue, 2-3 the l planes, 4 the FP64 sums.
// Every wait is bounded (1 s): a wait that gives up sets the status word and the roles wind down,
// the producer waiting for its loads in flight.
// ---------------------------------------------------------------------------------------------
constexpr int GTC_THREADS = 160;
constexpr int GTC_BAND = 4;                                  // rows of the contracted mode per band
constexpr int GTC_UNIT_BYTES = GTC_BAND * 24 * 128;          // 12 KB: one band of a tile
constexpr int GTC_SLOT_BYTES = 2 * GTC_UNIT_BYTES;           // the band and its l plane
constexpr int GTC_SLOTS = 8;
constexpr int GTC_PAD = 14 * 1024;                           // reach of the last MMA past the ring
constexpr int GTC_UNITS_PER_TILE = 2 * 24 / GTC_BAND;        // 6 bands of i, then 6 bands of j
constexpr int GTC_DRAIN_TILES = 1;                           // tiles per TMEM set before it is drained
constexpr size_t GTC_SMEM = 1024 + (size_t)GTC_SLOTS * GTC_SLOT_BYTES + GTC_PAD;

__device__ __forceinline__ void load_4d(const CUtensorMap* map, uint64_t* bar, void* dst, int x, int y, int z,
                                        int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
      "[%2];" ::"r"(tma::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tma::smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
      : "memory");
}

__global__ void __launch_bounds__(GTC_THREADS, 1)
    pair_gram_tc_kernel(const __grid_constant__ CUtensorMap map_i, const __grid_constant__ CUtensorMap map_j,
                        const PairGeom g, double* __restrict__ Ga, double* __restrict__ Gb, int* status) {
  extern __shared__ __align__(1024) uint8_t gtc_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(gtc_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[GTC_SLOTS], ready[GTC_SLOTS], empty[GTC_SLOTS], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int per = (int)((g.ntiles + gridDim.x - 1) / gridDim.x);
  const int t0 = (int)blockIdx.x * per;
  const int my_tiles = (g.ntiles > t0) ? min(per, (int)g.ntiles - t0) : 0;
  const int my_units = my_tiles * GTC_UNITS_PER_TILE;
  const int nsets = (my_tiles + GTC_DRAIN_TILES - 1) / GTC_DRAIN_TILES;  // TMEM set uses
  if (threadIdx.x == 0) {
    for (int i = 0; i < GTC_SLOTS; ++i) {
      tma::mbar_init(&full[i], 1);
      tma::mbar_init(&ready[i], 2);
      tma::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tma::mbar_init(&tfull[i], 1);
      tma::mbar_init(&tempty[i], 1);
    }
    tma::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tma::smem_u32(&tmem_base)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  const uint32_t tmem = tmem_base;  // set s at column 128 s: D_b, E_b, D_a, E_a at +0, +32, +64, +96

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int ca = (int)(t0 / g.ncb), ccb = (int)(t0 - (int64_t)ca * g.ncb), ub = 0;
      int issued = 0;
      bool ok = true;
      for (; ok && issued < my_units; ++issued) {
        const int slot = issued % GTC_SLOTS;
        const uint32_t ph = (uint32_t)((issued / GTC_SLOTS) & 1);
        if (issued >= GTC_SLOTS && !tma::mbar_wait(&empty[slot], ph ^ 1u, status)) {
          ok = false;
          break;
        }
        uint8_t* dst = base + (size_t)slot * GTC_SLOT_BYTES;
        tma::mbar_expect_tx(&full[slot], GTC_UNIT_BYTES);
        if (ub < 6)
          tma::load_3d(&map_i, &full[slot], dst, ccb * PCOLS, 0, ca * 24 + GTC_BAND * ub);
        else
          load_4d(&map_j, &full[slot], dst, ccb * PCOLS, 0, GTC_BAND * (ub - 6), ca);
        if (++ub == GTC_UNITS_PER_TILE) {
          ub = 0;
          if (++ccb == (int)g.ncb) {
            ccb = 0;
            ++ca;
          }
        }
      }
      if (!ok) {
        // let the loads in flight land before the CTA leaves (bounded, ignoring the status word)
        for (int q = max(issued - GTC_SLOTS, 0); q < issued; ++q) {
          const int sq = q % GTC_SLOTS;
          const uint32_t pp = (uint32_t)((q / GTC_SLOTS) & 1);
          const uint64_t tw = tma::gtimer();
          uint32_t okd = 0;
          while (!okd && tma::gtimer() - tw < DRAIN_NS) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(okd)
                : "r"(tma::smem_u32(&full[sq])), "r"(pp)
                : "memory");
          }
          if (!okd) break;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = tcg::idesc_tf32(128, 32);
      bool ok = true;
      int u = 0;
      for (int set = 0; ok && set < nsets; ++set) {
        const uint32_t acc = (uint32_t)(set & 1), aph = (uint32_t)((set >> 1) & 1);
        if (set >= 2 && !tma::mbar_wait(&tempty[acc], aph ^ 1u, status)) break;
        tcg::fence_after();
        const uint32_t dt = tmem + acc * 128u;
        const int uend = min(my_units, (set + 1) * GTC_DRAIN_TILES * GTC_UNITS_PER_TILE);
        bool first_b = true, first_a = true;
        for (; u < uend; ++u) {
          const int slot = u % GTC_SLOTS;
          const uint32_t ph = (uint32_t)((u / GTC_SLOTS) & 1);
          if (!tma::mbar_wait(&full[slot], ph, status) || !tma::mbar_wait(&ready[slot], ph, status)) {
            ok = false;
            break;
          }
          tcg::fence_after();
          const bool on_b = (u % GTC_UNITS_PER_TILE) < 6;
          const uint32_t hi = tma::smem_u32(base + (size_t)slot * GTC_SLOT_BYTES), lo = hi + GTC_UNIT_BYTES;
          const uint32_t dD = dt + (on_b ? 0u : 64u), dE = dD + 32u;
          bool& first = on_b ? first_b : first_a;
#pragma unroll
          for (int gr = 0; gr < GTC_BAND; ++gr)
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              const uint32_t off = (uint32_t)(gr * 3072 + 32 * k4);
              const uint64_t bh = tcg::sw128_desc(hi + off);
              const uint32_t accum = first ? 0u : 1u;
              tcg::mma_tf32(dD, tcg::sw128_desc(hi + off), bh, idesc, accum);
              tcg::mma_tf32(dE, tcg::sw128_desc(lo + off), bh, idesc, accum);
              first = false;
            }
          tcg::mma_commit(&empty[slot]);
        }
        if (!ok) break;
        tcg::mma_commit(&tfull[acc]);
      }
    }
  } else if (warp < 4) {
    // ---------------- l = x - (x with its 13 low mantissa bits cleared) ----------------
    const int t = (int)threadIdx.x - 64;  // 0..63
    for (int u = 0; u < my_units; ++u) {
      const int slot = u % GTC_SLOTS;
      const uint32_t ph = (uint32_t)((u / GTC_SLOTS) & 1);
      if (!tma::mbar_wait(&full[slot], ph, status)) break;
      const float4* src = reinterpret_cast<const float4*>(base + (size_t)slot * GTC_SLOT_BYTES);
      float4* dst = reinterpret_cast<float4*>(base + (size_t)slot * GTC_SLOT_BYTES + GTC_UNIT_BYTES);
      for (int q = t; q < GTC_UNIT_BYTES / 16; q += 64) {
        const float4 x = src[q];
        float4 l;
        l.x = x.x - __uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u);
        l.y = x.y - __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u);
        l.z = x.z - __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u);
        l.w = x.w - __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u);
        dst[q] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) tcg::mbar_arrive(&ready[slot]);
    }
  } else {
    // ---------------- FP64 sums of the TMEM sets (TMEM lanes 0..31 = rows 0..31) ----------------
    double fb[24], fa[24];
#pragma unroll
    for (int c = 0; c < 24; ++c) fb[c] = fa[c] = 0.0;
    for (int set = 0; set < nsets; ++set) {
      const uint32_t acc = (uint32_t)(set & 1), aph = (uint32_t)((set >> 1) & 1);
      if (!tma::mbar_wait(&tfull[acc], aph, status)) break;
      tcg::fence_after();
      const uint32_t dt = tmem + acc * 128u;
      float d[16], e[16];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        // columns 0..15 and 16..23 (16..31 loaded, the rest ignored) of D and E, for each Gram
        tcg::tmem_ld16(dt + 16u * half, d);
        tcg::tmem_ld16(dt + 32u + 16u * half, e);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (16 * half + c < 24) fb[16 * half + c] += (double)d[c] + 2.0 * (double)e[c];
        tcg::tmem_ld16(dt + 64u + 16u * half, d);
        tcg::tmem_ld16(dt + 96u + 16u * half, e);
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (16 * half + c < 24) fa[16 * half + c] += (double)d[c] + 2.0 * (double)e[c];
      }
      tcg::fence_before();
      __syncwarp();
      if (lane == 0) tcg::mbar_arrive(&tempty[acc]);
    }
    // G = (F + F^T) / 2 through shared memory (the ring is idle once every set is summed)
    double* Fs = reinterpret_cast<double*>(base);  // [2][24][24]
    if (lane < 24)
#pragma unroll
      for (int c = 0; c < 24; ++c) {
        Fs[lane * 24 + c] = fb[c];
        Fs[576 + lane * 24 + c] = fa[c];
      }
    __syncwarp();
    if (lane < 24)
      for (int c = lane; c < 24; ++c) {
        const double vb = 0.5 * (Fs[lane * 24 + c] + Fs[c * 24 + lane]);
        const double va = 0.5 * (Fs[576 + lane * 24 + c] + Fs[576 + c * 24 + lane]);
        atomicAdd(&Gb[lane * 24 + c], vb);
        atomicAdd(&Ga[lane * 24 + c], va);
        if (c != lane) {
          atomicAdd(&Gb[c * 24 + lane], vb);
          atomicAdd(&Ga[c * 24 + lane], va);
        }
      }
  }
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
}

// 4-D map of X[A][na][nb][B] that takes mode a before mode b: dims (B, na, nb, A), box (32, na, rows, 1);
// a tile band lands as rows (j, i).
bool make_map_pair_ji(CUtensorMap* m, const float* X, const PairGeom& g, int rows) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)g.B, (cuuint64_t)g.na, (cuuint64_t)g.nb, (cuuint64_t)g.A};
  cuuint64_t strides[3] = {(cuuint64_t)g.nb * (cuuint64_t)g.B * 4, (cuuint64_t)g.B * 4,
                           (cuuint64_t)g.na * (cuuint64_t)g.nb * (cuuint64_t)g.B * 4};
  cuuint32_t box[4] = {(cuuint32_t)PCOLS, (cuuint32_t)g.na, (cuuint32_t)rows, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(X), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3-D map of X[A][na][nb][B] as (B, nb, na * A), box (32, nb, rows): a whole tile (rows = na) or one band.
bool make_map_pair(CUtensorMap* m, const float* X, const PairGeom& g, int rows) {
  auto fn = tensor_map_encoder();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.B, (cuuint64_t)g.nb, (cuuint64_t)g.na * (cuuint64_t)g.A};
  cuuint64_t strides[2] = {(cuuint64_t)g.B * 4, (cuuint64_t)g.nb * (cuuint64_t)g.B * 4};
  cuuint32_t box[3] = {(cuuint32_t)PCOLS, (cuuint32_t)g.nb, (cuuint32_t)rows};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

PairGeom geom(int64_t A, int na, int nb, int64_t B) {
  PairGeom g;
  g.A = A;
  g.B = B;
  g.na = na;
  g.nb = nb;
  g.ncb = (B + PCOLS - 1) / PCOLS;
  g.ntiles = A * g.ncb;
  g.tile_bytes = (uint32_t)na * (uint32_t)nb * 128u;
  g.stage_bytes = (g.tile_bytes + 1023u) & ~1023u;
  return g;
}

int sm_count() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return std::max(nsm, 1);
}

ProjGeom proj_geom(const PairGeom& g, int RA, int RB) {
  ProjGeom pg;
  pg.ka = g.na >= 16 ? (g.na + 1) / 2 : g.na;
  pg.nbands = (g.na + pg.ka - 1) / pg.ka;
  pg.unit_bytes = (uint32_t)pg.ka * (uint32_t)g.nb * 128u;
  pg.stage_bytes = (pg.unit_bytes + 1023u) & ~1023u;
  const size_t fixed = 1024 + sizeof(float) * ((size_t)pg.ka * RB * PCOLS + (size_t)g.na * RA + (size_t)g.nb * RB);
  const size_t cap = 227 * 1024;
  pg.nst = cap > fixed ? (int)std::min<size_t>(PROJ_STAGES_MAX, (cap - fixed) / pg.stage_bytes) : 0;
  return pg;
}

size_t proj_smem(const PairGeom& g, const ProjGeom& pg, int RA, int RB) {
  return 1024 + (size_t)pg.nst * pg.stage_bytes +
         sizeof(float) * ((size_t)pg.ka * RB * PCOLS + (size_t)g.na * RA + (size_t)g.nb * RB);
}

template <int RA, int RB>
cudaError_t launch_proj(const float* X, const PairGeom& g, const double* Ua, int ra, int lda, const double* Ub,
                        int rb, int ldb, float* out, double* norm_in, double* norm_out, double* resid, int* status,
                        cudaStream_t s) {
  const ProjGeom pg = proj_geom(g, RA, RB);
  if (pg.nst < 2) return cudaErrorInvalidValue;
  CUtensorMap m;
  if (!make_map_pair(&m, X, g, pg.ka)) return cudaErrorInvalidValue;
  const size_t smem = proj_smem(g, pg, RA, RB);
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(pair_project_kernel<RA, RB>));
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(g.ntiles, sm_count());
  pair_project_kernel<RA, RB><<<grid, PROJ_THREADS, smem, s>>>(m, g, pg, Ua, ra, lda, Ub, rb, ldb, out, norm_in,
                                                               norm_out, resid, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_proj_ws(const float* X, const PairGeom& g, const double* Ua, int ra, int lda, const double* Ub,
                           int rb, int ldb, float* out, double* norm_in, double* norm_out, double* resid, int* status,
                           cudaStream_t s) {
  // two bands of 12 rows of mode a (na = 24), nb = 24
  if (g.na != 24 || g.nb != 24 || (g.B & 3) != 0) return cudaErrorInvalidValue;
  if (g.ntiles * 2 > 0x7fffffffll) return cudaErrorInvalidValue;  // 32-bit unit counters in the kernel
  ProjGeom pg;
  pg.ka = 12;
  pg.nbands = 2;
  pg.unit_bytes = (uint32_t)pg.ka * (uint32_t)g.nb * 128u;
  pg.stage_bytes = (pg.unit_bytes + 1023u) & ~1023u;
  const size_t fixed = 1024 + sizeof(float) * 3 * (size_t)pg.ka * 8 * PCOLS;  // three Z buffers
  const size_t cap = 227 * 1024;
  pg.nst = (int)std::min<size_t>(PROJ_STAGES_MAX, (cap - fixed) / pg.stage_bytes);
  if (pg.nst < 2) return cudaErrorInvalidValue;
  const size_t smem = fixed + (size_t)pg.nst * pg.stage_bytes;
  CUtensorMap m;
  if (!make_map_pair(&m, X, g, pg.ka)) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(pair_project_ws_kernel<24, 12>));
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(g.ntiles, sm_count());
  pair_project_ws_kernel<24, 12><<<grid, 32 * (pg.ka + WS_W2), smem, s>>>(m, g, pg, Ua, ra, lda, Ub, rb, ldb, out,
                                                                            norm_in, norm_out, resid, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

bool pair_gram_supported(int64_t A, int64_t na, int64_t nb, int64_t B) {
  return A >= 1 && na >= 1 && nb >= 1 && na <= PAIR_MAX_GRAM && nb <= PAIR_MAX_GRAM && B >= 4 && B % 4 == 0 &&
         na * A <= 0x7fffffffll && B <= 0x7fffffffll;
}

bool pair_project_supported(int64_t A, int64_t na, int64_t nb, int64_t B, int64_t ra, int64_t rb) {
  if (A < 1 || na < 1 || nb < 1 || na > PAIR_MAX_PROJ || nb > PAIR_MAX_PROJ || B < 4 || B % 4 != 0) return false;
  if (ra < 1 || rb < 1 || ra > 16 || rb > 16 || na * A > 0x7fffffffll || B > 0x7fffffffll) return false;
  if (rb * PCOLS > 2 * PROJ_THREADS) return false;
  const PairGeom g = geom(A, (int)na, (int)nb, B);
  return proj_geom(g, ra > 8 ? 16 : 8, rb > 8 ? 16 : 8).nst >= 2;
}

cudaError_t launch_pair_gram(const float* X, int64_t A, int na, int nb, int64_t B, double* Ga, double* Gb,
                             int* status, cudaStream_t s, bool tensor_cores) {
  if (!pair_gram_supported(A, na, nb, B) || (reinterpret_cast<uintptr_t>(X) & 15) != 0) return cudaErrorInvalidValue;
  const PairGeom g = geom(A, na, nb, B);
  CUtensorMap m;
  if (!make_map_pair(&m, X, g, na)) return cudaErrorInvalidValue;
  const int na8 = (na + 7) / 8, nb8 = (nb + 7) / 8;
  const int wa = na8 * (na8 + 1) / 2, wb = nb8 * (nb8 + 1) / 2;
  const int threads = 32 * (wa + wb);
  const size_t smem = 1024 + 2 * (size_t)g.stage_bytes + sizeof(double) * 64 * (size_t)(wa + wb);
  if (threads > 384 || smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(pair_gram_kernel));
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(g.ntiles, sm_count());
  const double K = (double)A * (double)B;  // columns per row of either unfolding, over the whole tensor
  ProfScope prof(K_PAIR_GRAM, s, (double)na * (na + 1) * K * nb + (double)nb * (nb + 1) * K * na,
                 4.0 * K * na * nb);
  if (tensor_cores && na == 24 && nb == 24 && g.ntiles <= 0x7fffffffll) {
    CUtensorMap mi, mj;
    if (make_map_pair(&mi, X, g, GTC_BAND) && make_map_pair_ji(&mj, X, g, GTC_BAND)) {
      e = allow_max_smem(reinterpret_cast<const void*>(pair_gram_tc_kernel));
      if (e != cudaSuccess) return e;
      pair_gram_tc_kernel<<<grid, GTC_THREADS, GTC_SMEM, s>>>(mi, mj, g, Ga, Gb, status);
      note_launch();
      return cudaGetLastError();
    }
  }
  if (na == 24 && nb == 24 && g.ntiles <= 0x7fffffffll) {
    const size_t smem24 = 1024 + G24_STAGES * (size_t)g.stage_bytes + sizeof(double) * 64 * 12;
    e = allow_max_smem(reinterpret_cast<const void*>(pair_gram24_kernel));
    if (e != cudaSuccess) return e;
    pair_gram24_kernel<<<grid, 384, smem24, s>>>(m, g, Ga, Gb, status);
    note_launch();
    return cudaGetLastError();
  }
  pair_gram_kernel<<<grid, threads, smem, s>>>(m, g, wa, Ga, Gb, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_pair_project(const float* X, int64_t A, int na, int nb, int64_t B, const double* Ua, int ra,
                                int lda, const double* Ub, int rb, int ldb, float* out, double* norm_in,
                                double* norm_out, double* resid, int* status, cudaStream_t s) {
  if (!pair_project_supported(A, na, nb, B, ra, rb) || (reinterpret_cast<uintptr_t>(X) & 15) != 0)
    return cudaErrorInvalidValue;
  const PairGeom g = geom(A, na, nb, B);
  const double elems = (double)A * na * nb * (double)B;
  ProfScope prof(K_PAIR_PROJ, s, 2.0 * elems * rb + 2.0 * (double)A * na * rb * (double)B * ra,
                 4.0 * elems + 4.0 * (double)A * ra * rb * (double)B);
  if (ra <= 8 && rb <= 8 && na == 24 && nb == 24) return launch_proj_ws(X, g, Ua, ra, lda, Ub, rb, ldb, out, norm_in, norm_out,
                                                            resid, status, s);
  if (ra <= 8 && rb <= 8) return launch_proj<8, 8>(X, g, Ua, ra, lda, Ub, rb, ldb, out, norm_in, norm_out, resid, status, s);
  if (ra <= 8) return launch_proj<8, 16>(X, g, Ua, ra, lda, Ub, rb, ldb, out, norm_in, norm_out, resid, status, s);
  if (rb <= 8) return launch_proj<16, 8>(X, g, Ua, ra, lda, Ub, rb, ldb, out, norm_in, norm_out, resid, status, s);
  return launch_proj<16, 16>(X, g, Ua, ra, lda, Ub, rb, ldb, out, norm_in, norm_out, resid, status, s);
}

}  // namespace bht

// tri.cu — the three innermost modes of a layer intermediate contracted in one read:
//   X viewed as [A][n1][n2][n3] (each slab of n1 n2 n3 fp32 contiguous),
//   out[A][r1][r2][r3] = X x_1 U1^T x_2 U2^T x_3 U3^T,
// eq. ht_leaf_contraction for three leaves at once (Step 1 of Algorithm 2 once the outer modes are
// contracted), with ||X||^2 and ||out||^2 for the skip test (the energy the pass removes).
//
// After the two-mode pass over the batch the intermediate is small (173 MB for 64 items of 24^5), and
// two more launches (a two-mode pass over the middle modes, then the innermost mode) each pay their fixed
// cost and part of a read. Here a persistent CTA per SM walks whole slabs (55 KB at 24^3) through a ring of
// three 1-D bulk copies (cp.async.bulk on an mbarrier, bounded waits), and contracts each slab in shared
// memory in three steps: the outermost mode over four adjacent columns per thread (16-byte reads, the basis
// entries broadcast), then the middle mode, then the innermost, which writes r1 r2 r3 values per slab.
// Products and sums in FP32 with round-to-nearest; the norms of each slab are added to double-single
// accumulators (Knuth's TwoSum) and folded into FP64 at the end.
#include <cstdint>

#include "internal.cuh"
#include "tma.cuh"

namespace bht {
namespace {

constexpr int TRI_GROUP = 192;  // threads of one slab group (six warps)
constexpr int TRI_STAGES = 3;
constexpr int TRI_MAX_N = 32;
constexpr int TRI_MAX_R = 8;
constexpr int TRI_MAX_SLAB = 13824;  // floats: three stages and two groups' work areas fit shared memory
constexpr uint64_t TRI_DRAIN_NS = 100000000ull;

struct TriGeom {
  int64_t A;
  int n1, n2, n3, r1, r2, r3;
  int n23, slab;          // n2 n3 and n1 n2 n3 (floats)
  int t1s;                // row stride of T1: n2 n3 padded to 24 mod 32 (the rows a and a + 1 of step 2's warps
                          // fall on disjoint banks)
  int n3p;                // row stride of T2: n3 padded to 3 mod 4 (odd for step 3's column reads; rows 8 apart
                          // on disjoint banks for step 2's writes)
  uint32_t slab_bytes;    // 4 slab
  uint32_t stage_bytes;   // slab_bytes rounded up to 128
};

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(tma::smem_u32(dst)), "l"(src), "r"(bytes), "r"(tma::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void two_sum(float v, float& hi, float& lo) {
  const float s = hi + v;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (v - bp);
  hi = s;
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(TRI_GROUP) : "memory");
}
// AND of v over the threads of a group, which also synchronises them
__device__ __forceinline__ bool group_and(int grp, bool v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n selp.s32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "r"(1 + grp), "r"(TRI_GROUP)
      : "memory");
  return r != 0;
}

// Two groups of TRI_GROUP threads take the CTA's slabs in turn (slab k to group k % 2), each with its own
// T1 and T2 and its own named barrier, so that one group's barrier waits overlap the other's arithmetic.
// The ring's stage k % 3 holds slab k; the group that consumed it refills it with slab k + 3 once its step 1
// has read it. A wait that gives up raises the abort flag; both groups leave at their next slab and thread
// 0 waits (bounded) for the loads still pending before the CTA exits.
// N1, N2, N3: the mode sizes at compile time (0: read from g), so that the hot shape's loops unroll.
template <int N1, int N2, int N3>
__global__ void __launch_bounds__(2 * TRI_GROUP, 1)
    tri_project_kernel(const float* __restrict__ X, const TriGeom g, const double* __restrict__ U1, int ld1,
                       const double* __restrict__ U2, int ld2, const double* __restrict__ U3, int ld3,
                       float* __restrict__ out, double* norm_in, double* norm_out, double* resid, int* status) {
  extern __shared__ __align__(128) uint8_t tsm[];
  const int t12 = TRI_MAX_R * g.t1s + ((TRI_MAX_R * TRI_MAX_R * g.n3p + 3) & ~3);  // T1 and T2 of one group
  float* work = reinterpret_cast<float*>(tsm + (size_t)TRI_STAGES * g.stage_bytes);
  float* B1 = work + 2 * t12;            // [n1][8][2]: each entry twice, for packed FMAs
  float* B2 = B1 + 2 * TRI_MAX_R * g.n1;  // [n2][8]
  float* B3 = B2 + TRI_MAX_R * g.n2;      // [n3][8]
  __shared__ __align__(8) uint64_t full[TRI_STAGES];
  __shared__ int pend[TRI_STAGES];       // 1 + the parity of a load issued into the stage and not yet consumed
  __shared__ int abort_flag;
  __shared__ double red[2 * (2 * TRI_GROUP / 32)];
  const int tid = threadIdx.x;
  const int grp = tid / TRI_GROUP, gt = tid - grp * TRI_GROUP;
  float* T1 = work + grp * t12;                  // [8][n23]
  float* T2 = T1 + TRI_MAX_R * g.t1s;            // [8][8][n3p]
  for (int e = tid; e < TRI_MAX_R * g.n1; e += blockDim.x) {
    const int i = e / TRI_MAX_R, a = e - i * TRI_MAX_R;
    const float u = a < g.r1 ? (float)U1[(int64_t)i * ld1 + a] : 0.f;
    B1[2 * e] = u;
    B1[2 * e + 1] = u;
  }
  for (int e = tid; e < TRI_MAX_R * g.n2; e += blockDim.x) {
    const int j = e / TRI_MAX_R, b = e - j * TRI_MAX_R;
    B2[e] = b < g.r2 ? (float)U2[(int64_t)j * ld2 + b] : 0.f;
  }
  for (int e = tid; e < TRI_MAX_R * g.n3; e += blockDim.x) {
    const int k = e / TRI_MAX_R, c = e - k * TRI_MAX_R;
    B3[e] = c < g.r3 ? (float)U3[(int64_t)k * ld3 + c] : 0.f;
  }
  const int64_t G = gridDim.x;
  const int64_t mine = (g.A > blockIdx.x) ? (g.A - 1 - blockIdx.x) / G + 1 : 0;  // this CTA's slabs
  auto issue = [&](int64_t q) {  // slab q of this CTA into stage q % 3
    const int sq = (int)(q % TRI_STAGES);
    pend[sq] = 1 + (int)((q / TRI_STAGES) & 1);
    tma::mbar_expect_tx(&full[sq], g.slab_bytes);
    bulk_load(tsm + (size_t)sq * g.stage_bytes, X + (blockIdx.x + q * G) * (int64_t)g.slab, g.slab_bytes, &full[sq]);
  };
  if (tid == 0) {
    for (int s = 0; s < TRI_STAGES; ++s) {
      tma::mbar_init(&full[s], 1);
      pend[s] = 0;
    }
    abort_flag = 0;
    tma::fence_mbar_init();
    for (int64_t q = 0; q < mine && q < TRI_STAGES; ++q) issue(q);
  }
  __syncthreads();

  float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
  const int n1 = N1 ? N1 : g.n1, n2 = N2 ? N2 : g.n2, n3 = N3 ? N3 : g.n3;
  const int n23 = (N2 && N3) ? N2 * N3 : g.n23;
  const int quads = n23 / 4;
  const int r13 = g.r1 * n3, r12 = g.r1 * g.r2;
  for (int64_t k = grp; k < mine; k += 2) {
    const int s = (int)(k % TRI_STAGES);
    const bool got = *(volatile int*)&abort_flag == 0 && tma::mbar_wait(&full[s], (uint32_t)((k / TRI_STAGES) & 1), status);
    if (!group_and(grp, got)) {
      if (gt == 0) abort_flag = 1;
      break;
    }
    if (gt == 0) pend[s] = 0;
    const int64_t slab = blockIdx.x + k * G;
    const float* Xs = reinterpret_cast<const float*>(tsm + (size_t)s * g.stage_bytes);
    // step 1: T1[a][q] = sum_i U1[i][a] X[i][q], four adjacent columns per thread (two packed pairs)
    float2 xxp = make_float2(0.f, 0.f);
    for (int qd = gt; qd < quads; qd += TRI_GROUP) {
      float2 acc[TRI_MAX_R][2];
#pragma unroll
      for (int a = 0; a < TRI_MAX_R; ++a) acc[a][0] = acc[a][1] = make_float2(0.f, 0.f);
#pragma unroll 8
      for (int i = 0; i < n1; ++i) {
        const float4 x = *reinterpret_cast<const float4*>(Xs + i * n23 + 4 * qd);
        const float2 x01 = make_float2(x.x, x.y), x23 = make_float2(x.z, x.w);
        xxp = ffma2(x01, x01, xxp);
        xxp = ffma2(x23, x23, xxp);
        const float4* ud = reinterpret_cast<const float4*>(B1 + i * 2 * TRI_MAX_R);
#pragma unroll
        for (int a2 = 0; a2 < TRI_MAX_R / 2; ++a2) {
          const float4 u = ud[a2];  // (u_a, u_a, u_a+1, u_a+1), a = 2 a2
          const float2 ua = make_float2(u.x, u.y), ub = make_float2(u.z, u.w);
          acc[2 * a2][0] = ffma2(x01, ua, acc[2 * a2][0]);
          acc[2 * a2][1] = ffma2(x23, ua, acc[2 * a2][1]);
          acc[2 * a2 + 1][0] = ffma2(x01, ub, acc[2 * a2 + 1][0]);
          acc[2 * a2 + 1][1] = ffma2(x23, ub, acc[2 * a2 + 1][1]);
        }
      }
#pragma unroll
      for (int a = 0; a < TRI_MAX_R; ++a)
        *reinterpret_cast<float4*>(T1 + a * g.t1s + 4 * qd) = make_float4(acc[a][0].x, acc[a][0].y, acc[a][1].x, acc[a][1].y);
    }
    two_sum(xxp.x + xxp.y, xh, xl);
    group_sync(grp);  // T1 complete; the stage is free
    if (gt == 0 && k + TRI_STAGES < mine) issue(k + TRI_STAGES);
    // step 2: T2[a][b][kk] = sum_j U2[j][b] T1[a][j][kk]
    for (int it = gt; it < r13; it += TRI_GROUP) {
      const int a = it / n3, kk = it - a * n3;
      float acc[TRI_MAX_R];
#pragma unroll
      for (int b = 0; b < TRI_MAX_R; ++b) acc[b] = 0.f;
      const float* t1 = T1 + a * g.t1s + kk;
#pragma unroll 8
      for (int j = 0; j < n2; ++j) {
        const float t = t1[j * n3];
        const float4 u0 = *reinterpret_cast<const float4*>(B2 + j * TRI_MAX_R);
        const float4 u1 = *reinterpret_cast<const float4*>(B2 + j * TRI_MAX_R + 4);
        acc[0] = fmaf(t, u0.x, acc[0]);
        acc[1] = fmaf(t, u0.y, acc[1]);
        acc[2] = fmaf(t, u0.z, acc[2]);
        acc[3] = fmaf(t, u0.w, acc[3]);
        acc[4] = fmaf(t, u1.x, acc[4]);
        acc[5] = fmaf(t, u1.y, acc[5]);
        acc[6] = fmaf(t, u1.z, acc[6]);
        acc[7] = fmaf(t, u1.w, acc[7]);
      }
#pragma unroll
      for (int b = 0; b < TRI_MAX_R; ++b) T2[(a * TRI_MAX_R + b) * g.n3p + kk] = acc[b];
    }
    group_sync(grp);  // T2 complete; T1 free
    // step 3: out[a][b][c] = sum_kk U3[kk][c] T2[a][b][kk]; item it = 2 (a r2 + b) + h sums the kk of
    // parity h, and the pair of lanes (h = 0, 1) adds its halves through a shuffle
    float yy = 0.f;
    for (int base = 0; base < 2 * r12; base += TRI_GROUP) {
      const int it = base + gt;
      const bool act = it < 2 * r12;
      const int ab = it >> 1, h = it & 1;
      float acc[TRI_MAX_R];
#pragma unroll
      for (int c = 0; c < TRI_MAX_R; ++c) acc[c] = 0.f;
      if (act) {
        const int a = ab / g.r2, b = ab - a * g.r2;
        const float* t2 = T2 + (a * TRI_MAX_R + b) * g.n3p;
#pragma unroll 4
        for (int kk = h; kk < n3; kk += 2) {
          const float t = t2[kk];
          const float4 u0 = *reinterpret_cast<const float4*>(B3 + kk * TRI_MAX_R);
          const float4 u1 = *reinterpret_cast<const float4*>(B3 + kk * TRI_MAX_R + 4);
          acc[0] = fmaf(t, u0.x, acc[0]);
          acc[1] = fmaf(t, u0.y, acc[1]);
          acc[2] = fmaf(t, u0.z, acc[2]);
          acc[3] = fmaf(t, u0.w, acc[3]);
          acc[4] = fmaf(t, u1.x, acc[4]);
          acc[5] = fmaf(t, u1.y, acc[5]);
          acc[6] = fmaf(t, u1.z, acc[6]);
          acc[7] = fmaf(t, u1.w, acc[7]);
        }
      }
#pragma unroll
      for (int c = 0; c < TRI_MAX_R; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
      if (act && h == 0) {
        float* o = out + (slab * r12 + ab) * g.r3;  // [slab][a][b][c], ab = a r2 + b
#pragma unroll
        for (int c = 0; c < TRI_MAX_R; ++c)
          if (c < g.r3) {
            o[c] = acc[c];
            yy = fmaf(acc[c], acc[c], yy);
          }
      }
    }
    two_sum(yy, yh, yl);
  }
  __syncthreads();
  if (tid == 0 && abort_flag) {
    // loads issued and not consumed: wait for them (bounded) so that none lands after the CTA has left
    for (int sq = 0; sq < TRI_STAGES; ++sq) {
      if (!pend[sq]) continue;
      const uint32_t par = (uint32_t)(pend[sq] - 1);
      const uint64_t t0 = tma::gtimer();
      uint32_t ok = 0;
      while (!ok && tma::gtimer() - t0 < TRI_DRAIN_NS) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(tma::smem_u32(&full[sq])), "r"(par)
            : "memory");
      }
    }
  }
  // the CTA's norms: warp sums, then thread 0
  double sx = (double)xh + (double)xl, sy = (double)yh + (double)yl;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  const int w = tid >> 5, l = tid & 31, nw = (int)(blockDim.x >> 5);
  if (l == 0) {
    red[w] = sx;
    red[nw + w] = sy;
  }
  __syncthreads();
  if (tid == 0) {
    double tx = 0.0, ty = 0.0;
    for (int q = 0; q < nw; ++q) {
      tx += red[q];
      ty += red[nw + q];
    }
    if (norm_in) atomicAdd(norm_in, tx);
    if (norm_out) atomicAdd(norm_out, ty);
    if (resid) atomicAdd(resid, tx - ty);
  }
}

size_t tri_smem(const TriGeom& g) {
  const size_t t12 = (size_t)TRI_MAX_R * g.t1s + (((size_t)TRI_MAX_R * TRI_MAX_R * g.n3p + 3) & ~(size_t)3);
  return (size_t)TRI_STAGES * g.stage_bytes +
         sizeof(float) * (2 * t12 + (size_t)TRI_MAX_R * (2 * g.n1 + g.n2 + g.n3));
}

}  // namespace

bool tri_project_supported(int64_t A, int64_t n1, int64_t n2, int64_t n3, int64_t r1, int64_t r2, int64_t r3) {
  if (A < 1 || n1 < 1 || n2 < 1 || n3 < 1 || n1 > TRI_MAX_N || n2 > TRI_MAX_N || n3 > TRI_MAX_N) return false;
  if (r1 < 1 || r2 < 1 || r3 < 1 || r1 > TRI_MAX_R || r2 > TRI_MAX_R || r3 > TRI_MAX_R) return false;
  const int64_t slab = n1 * n2 * n3;
  if ((n2 * n3) % 4 != 0 || slab > TRI_MAX_SLAB || A > ((int64_t)1 << 40) / slab) return false;
  // shared memory: the ring, both groups' T1 and T2, the bases (the opt-in maximum less static use)
  const int64_t stage = (4 * slab + 127) & ~(int64_t)127;
  const int64_t t1s = n2 * n3 + ((24 - (n2 * n3) % 32 + 32) % 32), n3p = n3 + ((3 - n3 % 4 + 4) % 4);
  const int64_t t12 = TRI_MAX_R * t1s + ((TRI_MAX_R * TRI_MAX_R * n3p + 3) & ~(int64_t)3);
  return TRI_STAGES * stage + 4 * (2 * t12 + TRI_MAX_R * (2 * n1 + n2 + n3)) <= 220 * 1024;
}

cudaError_t launch_tri_project(const float* X, int64_t A, int n1, int n2, int n3, const double* U1, int r1, int ld1,
                               const double* U2, int r2, int ld2, const double* U3, int r3, int ld3, float* out,
                               double* norm_in, double* norm_out, double* resid, int* status, cudaStream_t s) {
  if (!tri_project_supported(A, n1, n2, n3, r1, r2, r3) || (reinterpret_cast<uintptr_t>(X) & 15) != 0)
    return cudaErrorInvalidValue;
  TriGeom g;
  g.A = A;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.r1 = r1;
  g.r2 = r2;
  g.r3 = r3;
  g.n23 = n2 * n3;
  g.t1s = g.n23 + ((24 - g.n23 % 32 + 32) % 32);
  g.n3p = n3 + ((3 - n3 % 4 + 4) % 4);
  g.slab = n1 * n2 * n3;
  g.slab_bytes = (uint32_t)(sizeof(float) * g.slab);
  g.stage_bytes = (g.slab_bytes + 127u) & ~127u;
  const size_t sm = tri_smem(g);
  const bool hot = n1 == 24 && n2 == 24 && n3 == 24;
  const auto kern = hot ? tri_project_kernel<24, 24, 24> : tri_project_kernel<0, 0, 0>;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 2 * TRI_GROUP, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = (int)std::min<int64_t>(A, nsm);
  const double cols = (double)A;
  ProfScope prof(K_TRI_PROJ, s,
                 2.0 * cols * ((double)g.slab * r1 + (double)r1 * n2 * n3 * r2 + (double)r1 * r2 * n3 * r3),
                 4.0 * cols * ((double)g.slab + (double)r1 * r2 * r3));
  kern<<<grid, 2 * TRI_GROUP, sm, s>>>(X, g, U1, ld1, U2, ld2, U3, ld3, out, norm_in, norm_out, resid, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

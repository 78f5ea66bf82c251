// dense.cu — FP64 SIMT kernels of the plain path: Gram matrices of mode
// unfoldings, mode products (TTM), norms, small FP64 GEMMs and copies.
//
// Every full-data contraction of BHT-l2r (Algorithm 1) and HT-RISE
// (Algorithm 2) is one of two shapes over a view [A][I][B] of a layer
// intermediate (Section 2.1 unfolding of the node's index I):
//   Gram : G = X_(I) X_(I)^T                      (the SVD of eq. ht_leaf_svd
//          is taken through the eigenvectors of this Gram matrix)
//   TTM  : X x_I M, M = U^T to project (eq. ht_leaf_contraction) or M = U to
//          expand (eq. htucker_reconstruction).
// GB300 has few FP64 units (≈1/64 of the FP32 rate), so these kernels are
// FP64-ALU bound; they are the reference GPU form the mixed path is measured
// against.
#include <algorithm>

#include "internal.cuh"

namespace bht {

namespace {

constexpr int TILE = 64;   // output tile edge
constexpr int BK = 16;     // depth of one shared-memory stage
constexpr int NT = 256;    // threads per CTA (16 x 16, each 4 x 4 outputs)


// ---------------------------------------------------------------------------
// Gram of the middle index of X[A][I][B]
// grid.x: upper-triangular tile pairs (ti <= tj), grid.y: chunks of the
// flattened column index k = a * B + b.
// ---------------------------------------------------------------------------
template <typename T, typename Acc>
__global__ void __launch_bounds__(NT) gram_simt_kernel(const T* __restrict__ X, double* __restrict__ G,
                                                      int64_t A, int64_t I, int64_t B,
                                                      int64_t kchunk, int ntiles) {
  __shared__ Acc Xi[BK][TILE + 1];
  __shared__ Acc Xj[BK][TILE + 1];
  // decode the tile pair (ti, tj), ti <= tj, from blockIdx.x
  int pid = blockIdx.x, ti = 0;
  while (pid >= ntiles - ti) { pid -= ntiles - ti; ++ti; }
  const int tj = ti + pid;
  const int64_t i0 = (int64_t)ti * TILE, j0 = (int64_t)tj * TILE;
  const int64_t K = A * B;
  const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool along_k = B >= 8;
  // per-stage partial sums in Acc, folded into FP64 after every stage of BK columns
  double acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // load BK x TILE slabs of rows i0.. and j0..
    for (int e = threadIdx.x; e < BK * TILE; e += NT) {
      int kk, ii;
      if (along_k) { kk = e % BK; ii = e / BK; } else { ii = e % TILE; kk = e / TILE; }
      const int64_t k = k0 + kk;
      Acc vi = Acc(0), vj = Acc(0);
      if (k < kend) {
        const int64_t a = k / B, b = k - a * B;
        const int64_t base = a * I * B + b;
        if (i0 + ii < I) vi = static_cast<Acc>(X[base + (i0 + ii) * B]);
        if (ti != tj && j0 + ii < I) vj = static_cast<Acc>(X[base + (j0 + ii) * B]);
      }
      Xi[kk][ii] = vi;
      if (ti != tj) Xj[kk][ii] = vj;
    }
    __syncthreads();
    const Acc (*Bj)[TILE + 1] = (ti == tj) ? Xi : Xj;
    Acc part[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) part[u][v] = Acc(0);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Xi[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bj[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) part[u][v] = fma(a[u], b[v], part[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += static_cast<double>(part[u][v]);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t i = i0 + ty + 16 * u;
    if (i >= I) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t j = j0 + tx + 16 * v;
      if (j >= I) continue;
      if (ti == tj) {
        atomicAdd(G + i * I + j, acc[u][v]);
      } else {
        atomicAdd(G + i * I + j, acc[u][v]);
        atomicAdd(G + j * I + i, acc[u][v]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Gram of a short middle index (I <= 64) over a long column index: HBM-bound, so
// the column chunks are read once, coalesced, by persistent CTAs. A chunk holds
// CHC consecutive columns k = a * B + b: CHC values of b inside one a when
// B >= CHC, CHC / B whole slabs when B < CHC, CHC consecutive a when B == 1. It
// is staged transposed, Xs[c][i], so four consecutive i are one 16-byte
// shared load, by 4-byte asynchronous copies into one of two buffers while the
// other is read (each thread walks its elements of a chunk with a
// mixed-radix counter: no division per element). Thread (tile, group)
// accumulates the 4 x 4 block (ti, tj), ti <= tj, of G over the chunk columns
// of its group in FP32; the FP32 partials are added to FP64 registers every
// GRAM_FOLD chunks, summed over the groups at the end and added to G with FP64
// atomics (both triangles).
// ---------------------------------------------------------------------------
constexpr int CHC = 128;
constexpr int GRAM_FOLD = 2;
constexpr int GRAM_SMALL_THREADS = 256;

__device__ __forceinline__ void cp_async_f32(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// The elements of one chunk a thread copies: (al, i, b) of the chunk's slab al, row i, column b,
// visited as e = tid, tid + 256, ... of e = (al * I + i) * nb + b, advanced without division.
struct ChunkWalk {
  int b0, i0, al0;      // decomposition of tid
  int db, di, dal;      // of the step 256 (b carries into i, i into al)
  __device__ void init(int tid, int nb, int I) {
    b0 = tid % nb;
    const int t = tid / nb;
    i0 = t % I;
    al0 = t / I;
    db = GRAM_SMALL_THREADS % nb;
    const int tq = GRAM_SMALL_THREADS / nb;
    di = tq % I;
    dal = tq / I;
  }
};

__global__ void __launch_bounds__(GRAM_SMALL_THREADS) gram_small_kernel(const float* __restrict__ X, int64_t A,
                                                                        int I, int64_t B, double* __restrict__ G) {
  const int Ip = (I + 3) & ~3, T4 = Ip / 4, ntiles = T4 * (T4 + 1) / 2;
  const int groups = max(1, (int)blockDim.x / ntiles);
  extern __shared__ __align__(16) float gs[];  // Xs[2][CHC][Ip], then the FP64 reduction area
  const int tid = threadIdx.x;
  const int tile = tid % ntiles, grp = tid / ntiles;
  const bool active = grp < groups;
  int ti = 0, tj = 0;
  {
    int t = tile;
    while (t >= T4 - ti) { t -= T4 - ti; ++ti; }
    tj = ti + t;
  }
  // chunk geometry
  int64_t nb, na;
  if (B == 1) { nb = 1; na = CHC; }
  else if (B >= CHC) { nb = CHC; na = 1; }
  else { nb = B; na = CHC / B; }
  const int64_t chunks_b = (B == 1) ? 1 : (B + nb - 1) / nb;      // chunks along b in one slab group
  const int64_t groups_a = (A + na - 1) / na;
  const int64_t nchunks = groups_a * chunks_b;
  // zero both buffers once: the copies never write rows i >= I
  for (int e = tid; e < 2 * CHC * Ip; e += blockDim.x) gs[e] = 0.f;
  __syncthreads();
  ChunkWalk w;
  w.init(tid, (int)nb, I);
  const int nbi = (int)nb;
  auto stage = [&](int64_t ch, float* Xs) {
    if (ch < nchunks) {
      const int64_t ga = ch / chunks_b, gb = ch - ga * chunks_b;
      const int64_t a0 = ga * na, b0 = gb * nb;
      const int nah = (int)min(na, A - a0), nbh = (int)min(nb, B - b0);
      const float* src = X + (a0 * I) * B + b0;
      int b = w.b0, i = w.i0, al = w.al0;
      while (al < nah) {
        if (b < nbh) cp_async_f32(Xs + (al * nbi + b) * Ip + i, src + ((int64_t)al * I + i) * B + b);
        b += w.db;
        int carry = 0;
        if (b >= nbi) { b -= nbi; carry = 1; }
        i += w.di + carry;
        al += w.dal;
        if (i >= I) { i -= I; ++al; }
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  double acc64[4][4];
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc64[u][v] = 0.0; acc[u][v] = 0.f; }
  int since = 0;
  int buf = 0;
  stage(blockIdx.x, gs);
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    stage(ch + gridDim.x, gs + (buf ^ 1) * CHC * Ip);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    const float* Xs = gs + buf * CHC * Ip;
    const int64_t ga = ch / chunks_b, gb = ch - ga * chunks_b;
    const int64_t a0 = ga * na, b0 = gb * nb;
    const int ncol = (int)(min(na, A - a0) * min(nb, B - b0));
    if (active) {
      for (int c = grp; c < ncol; c += groups) {
        const float4 x = *reinterpret_cast<const float4*>(Xs + c * Ip + 4 * ti);
        const float4 y = *reinterpret_cast<const float4*>(Xs + c * Ip + 4 * tj);
        const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xa[u], ya[v], acc[u][v]);
      }
      if (++since == GRAM_FOLD) {
        since = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) { acc64[u][v] += (double)acc[u][v]; acc[u][v] = 0.f; }
      }
    }
    __syncthreads();  // this buffer is refilled by the next iteration's copies
    buf ^= 1;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc64[u][v] += (double)acc[u][v];
  // sum over the groups in shared memory (FP64), then one atomic per entry per CTA
  __syncthreads();
  double* red = reinterpret_cast<double*>(gs);  // [ntiles][16]
  for (int e = tid; e < ntiles * 16; e += blockDim.x) red[e] = 0.0;
  __syncthreads();
  if (active) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) atomicAdd(&red[tile * 16 + u * 4 + v], acc64[u][v]);
  }
  __syncthreads();
  for (int e = tid; e < ntiles * 16; e += blockDim.x) {
    const int tl = e / 16, u = (e / 4) % 4, v = e % 4;
    int a_ = 0, t = tl;
    while (t >= T4 - a_) { t -= T4 - a_; ++a_; }
    const int b_ = a_ + t;
    const int i = 4 * a_ + u, j = 4 * b_ + v;
    if (i >= I || j >= I) continue;
    const double val = red[e];
    if (val == 0.0) continue;
    atomicAdd(&G[(int64_t)i * I + j], val);
    if (a_ != b_) atomicAdd(&G[(int64_t)j * I + i], val);
  }
}

// ---------------------------------------------------------------------------
// TTM: out[a][s][b] = sum_t M(s,t) X[a][t][b]
// grid.x: tiles of the flattened column c = a * B + b, grid.y: tiles of s.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tout, typename Acc, typename Tm>
__global__ void __launch_bounds__(NT) ttm_simt_kernel(const Tin* __restrict__ X, Tout* __restrict__ out,
                                                      const Tm* __restrict__ M, int64_t ms, int64_t mt,
                                                      int64_t A, int64_t T, int64_t B, int64_t S, int64_t R2,
                                                      int64_t S_store, double* __restrict__ resid) {
  constexpr int PER = BK * TILE / NT;  // staged X elements per thread
  // rows padded to TILE + 4: 16-byte aligned for the vector reads of the product, and a stage written
  // along k spreads over the banks
  __shared__ __align__(16) Acc Ms[BK][TILE + 4];
  __shared__ __align__(16) Acc Xs[BK][TILE + 4];
  const int64_t c0 = (int64_t)blockIdx.x * TILE;
  const int64_t s0 = (int64_t)blockIdx.y * TILE;
  const int64_t AB = A * B;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool m_along_s = (ms == 1);
  const bool x_along_c = B >= 8;
  // the column c = a * B + b of every staged X element, and the output index s of every staged M
  // element, are fixed across the T stages
  int xkk[PER], xcc[PER], mkk[PER], mss[PER];
  int64_t xoff[PER], moff[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * NT;
    if (x_along_c) { xcc[q] = e % TILE; xkk[q] = e / TILE; } else { xkk[q] = e % BK; xcc[q] = e / BK; }
    const int64_t c = c0 + xcc[q];
    const int64_t a = c / B, b = c - a * B;
    xoff[q] = (c < AB) ? a * T * B + b : -1;
    if (m_along_s) { mss[q] = e % TILE; mkk[q] = e / TILE; } else { mkk[q] = e % BK; mss[q] = e / BK; }
    const int64_t sidx = s0 + mss[q];
    moff[q] = (sidx < S) ? sidx * ms : -1;
  }
  Acc acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = Acc(0);

  // the next stage's operands are loaded into registers while the current one is multiplied
  Acc xr[PER], mr[PER];
  auto fetch = [&](int64_t t0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int64_t tx_ = t0 + xkk[q], tm_ = t0 + mkk[q];
      xr[q] = (tx_ < T && xoff[q] >= 0) ? static_cast<Acc>(X[xoff[q] + tx_ * B]) : Acc(0);
      mr[q] = (tm_ < T && moff[q] >= 0) ? static_cast<Acc>(M[moff[q] + tm_ * mt]) : Acc(0);
    }
  };
  fetch(0);
  for (int64_t t0 = 0; t0 < T; t0 += BK) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      Xs[xkk[q]][xcc[q]] = xr[q];
      Ms[mkk[q]][mss[q]] = mr[q];
    }
    __syncthreads();
    if (t0 + BK < T) fetch(t0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Ms[kk][4 * ty + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Xs[kk][4 * tx + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double rq = 0.0;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int64_t c = c0 + 4 * tx + v;
    if (c >= AB) continue;
    const int64_t a = c / B, b = c - a * B;
    // B > 1: out[a][s][b]; B == 1: the new axis goes in front of the last R2 rows
    const int64_t o = a / R2, i = a - o * R2;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t sidx = s0 + 4 * ty + u;
      if (sidx < S_store) {
        const int64_t off = (B > 1) ? (a * S_store + sidx) * B + b : (o * S_store + sidx) * R2 + i;
        out[off] = static_cast<Tout>(acc[u][v]);
      } else if (sidx < S) {
        rq += (double)acc[u][v] * (double)acc[u][v];
      }
    }
  }
  if (resid) {
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) rq += __shfl_xor_sync(0xffffffffu, rq, o2);
    if ((threadIdx.x & 31) == 0 && rq != 0.0) atomicAdd(resid, rq);
  }
}

// ---------------------------------------------------------------------------
// Generic FP64 GEMM with strided operands. FP64 issues at about two FMA per
// clock per SM on this part, so the tile edge follows the output size (64, 32
// or 16, 256 threads each with (TE/16)^2 outputs) and K is split across CTAs
// until the grid covers every SM several times; grid.z splits K into chunks of
// kchunk and, with more than one chunk, every CTA adds alpha * its partial
// product to C atomically (C was scaled by beta beforehand).
// ---------------------------------------------------------------------------
template <int TE>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(int64_t M, int64_t N, int64_t K, double alpha,
                                                      const double* __restrict__ Am, int64_t a_rs, int64_t a_cs,
                                                      const double* __restrict__ Bm, int64_t b_rs, int64_t b_cs,
                                                      double beta, double* __restrict__ C, int64_t c_rs,
                                                      int64_t c_cs, int64_t kchunk) {
  constexpr int R = TE / 16;  // outputs per thread along each edge
  __shared__ double As[BK][TE + 1];
  __shared__ double Bs[BK][TE + 1];
  const int64_t m0 = (int64_t)blockIdx.y * TE, n0 = (int64_t)blockIdx.x * TE;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[R][R];
#pragma unroll
  for (int u = 0; u < R; ++u)
#pragma unroll
    for (int v = 0; v < R; ++v) acc[u][v] = 0.0;
  const bool a_along_m = (a_rs == 1);
  const bool b_along_n = (b_cs == 1);
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  K = min(K, kbeg + kchunk);
  for (int64_t k0 = kbeg; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BK * TE; e += NT) {
      int kk, mm;
      if (a_along_m) { mm = e % TE; kk = e / TE; } else { kk = e % BK; mm = e / BK; }
      const int64_t k = k0 + kk, m = m0 + mm;
      As[kk][mm] = (k < K && m < M) ? Am[m * a_rs + k * a_cs] : 0.0;
    }
    for (int e = threadIdx.x; e < BK * TE; e += NT) {
      int kk, nn;
      if (b_along_n) { nn = e % TE; kk = e / TE; } else { kk = e % BK; nn = e / BK; }
      const int64_t k = k0 + kk, n = n0 + nn;
      Bs[kk][nn] = (k < K && n < N) ? Bm[k * b_rs + n * b_cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[R], b[R];
#pragma unroll
      for (int u = 0; u < R; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < R; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int64_t m = m0 + ty + 16 * u;
    if (m >= M) continue;
#pragma unroll
    for (int v = 0; v < R; ++v) {
      const int64_t n = n0 + tx + 16 * v;
      if (n >= N) continue;
      double* cp = C + m * c_rs + n * c_cs;
      if (gridDim.z > 1)
        atomicAdd(cp, alpha * acc[u][v]);
      else
        *cp = (beta == 0.0) ? alpha * acc[u][v] : alpha * acc[u][v] + beta * (*cp);
    }
  }
}

// y(m) = alpha sum_k A(m, k) x(k) + beta y(m): one warp per output row.
__global__ void gemv_f64_kernel(int64_t M, int64_t K, double alpha, const double* __restrict__ Am, int64_t a_rs,
                                int64_t a_cs, const double* __restrict__ x, int64_t x_s, double beta,
                                double* __restrict__ y, int64_t y_s) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < M; m += nw) {
    double dot = 0.0;
    for (int64_t k = lane; k < K; k += 32) dot = fma(Am[m * a_rs + k * a_cs], x[k * x_s], dot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if (lane == 0) y[m * y_s] = (beta == 0.0) ? alpha * dot : alpha * dot + beta * y[m * y_s];
  }
}

// ---------------------------------------------------------------------------
// Reductions and copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void sqnorm_kernel(const T* __restrict__ x, int64_t n, double* __restrict__ acc) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = static_cast<double>(x[i]);
    s = fma(v, v, s);
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) atomicAdd(acc, s);
  }
}

// ||x||^2 of fp32 data at the FP32 rate with FP64-class accuracy: each square is split exactly into
// p + e (p = x*x rounded, e = fma(x, x, -p)) and added to a double-single accumulator (hi, lo) by
// Knuth's TwoSum, so the FP64 units (1/64 of the FP32 rate here) only see one value per thread.
__device__ __forceinline__ void ds_add_sq(float x, float& hi, float& lo) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  const float s = hi + p;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += err + e;
}

__global__ void sqnorm_f32_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ acc) {
  float hi = 0.f, lo = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // scalar head up to a 16-byte boundary, float4 body, scalar tail
  const int64_t head = std::min<int64_t>(n, (int64_t)(((16 - (reinterpret_cast<uintptr_t>(x) & 15)) & 15) / 4));
  if (tid < head) ds_add_sq(x[tid], hi, lo);
  const int64_t n4 = (n - head) / 4;
  const float4* x4 = reinterpret_cast<const float4*>(x + head);
  for (int64_t i = tid; i < n4; i += stride) {
    const float4 v = x4[i];
    ds_add_sq(v.x, hi, lo);
    ds_add_sq(v.y, hi, lo);
    ds_add_sq(v.z, hi, lo);
    ds_add_sq(v.w, hi, lo);
  }
  for (int64_t i = head + 4 * n4 + tid; i < n; i += stride) ds_add_sq(x[i], hi, lo);
  double s = (double)hi + (double)lo;
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) atomicAdd(acc, s);
  }
}

__global__ void trace_kernel(const double* __restrict__ G, int64_t n, double* __restrict__ acc) {
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += G[i * n + i];
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) atomicAdd(acc, s);
  }
}

template <typename Tin, typename Tout>
__global__ void copy_pad3_kernel(const Tin* __restrict__ in, int64_t A1, int64_t B1, int64_t C1,
                                 Tout* __restrict__ out, int64_t A2, int64_t B2, int64_t C2) {
  const int64_t total = A2 * B2 * C2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % C2;
    const int64_t ab = e / C2;
    const int64_t b = ab % B2, a = ab / B2;
    Tout v = Tout(0);
    if (a < A1 && b < B1 && c < C1) v = static_cast<Tout>(in[(a * B1 + b) * C1 + c]);
    out[e] = v;
  }
}

__global__ void copy_cols_kernel(const double* __restrict__ in, int64_t ld_in, int64_t rows, int64_t cols,
                                 double* __restrict__ out, int64_t ld_out) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    out[i * ld_out + j] = in[i * ld_in + j];
  }
}

template <typename Tin, typename Tout>
__global__ void cast_kernel(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = static_cast<Tout>(in[i]);
}

// fp32 -> FP64 four values at a time: one 16-byte load and two 16-byte stores per thread and step
__global__ void cast_f32_f64_vec_kernel(const float4* __restrict__ in, double2* __restrict__ out, int64_t n4) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 v = in[i];
    out[2 * i] = make_double2((double)v.x, (double)v.y);
    out[2 * i + 1] = make_double2((double)v.z, (double)v.w);
  }
}

__global__ void scale_cols_invsqrt_kernel(double* __restrict__ W, int64_t rows, int64_t cols,
                                          const double* __restrict__ lam) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e % cols;
    W[e] /= sqrt(fmax(lam[j], 1e-300));
  }
}

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014) of seed + index, mapped to [-1, 1)
__global__ void fill_uniform_kernel(double* __restrict__ X, int64_t n, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    X[e] = (double)(int64_t)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

// Unit column for every coordinate j = i * rb + k of a grown merged index with i >= ra0 or k >= rb0,
// numbered in C order from column col0: Q[j * ldq + col0 + idx(j)] = 1.
__global__ void unit_cols_kernel(double* __restrict__ Q, int64_t ldq, int64_t col0, int64_t ra0, int64_t rb0,
                                 int64_t ra, int64_t rb) {
  const int64_t total = ra * rb;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = j / rb, k = j - i * rb;
    int64_t idx;
    if (i < ra0) {
      if (k < rb0) continue;
      idx = i * (rb - rb0) + (k - rb0);
    } else {
      idx = ra0 * (rb - rb0) + (i - ra0) * rb + k;
    }
    Q[j * ldq + col0 + idx] = 1.0;
  }
}

__global__ void scale_strided_kernel(double* __restrict__ C, int64_t M, int64_t N, int64_t c_rs, int64_t c_cs,
                                     double beta) {
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double* cp = C + (e / N) * c_rs + (e % N) * c_cs;
    *cp = (beta == 0.0) ? 0.0 : beta * (*cp);
  }
}

__global__ void cast_matrix_kernel(const double* __restrict__ U, int64_t ms, int64_t mt, int64_t S, int64_t T,
                                   float* __restrict__ out) {
  const int64_t total = S * T;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sidx = e / T, t = e - sidx * T;
    out[e] = static_cast<float>(U[sidx * ms + t * mt]);
  }
}

__global__ void fill_identity_kernel(double* __restrict__ A, int64_t n) {
  const int64_t total = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    A[e] = (e / n == e % n) ? 1.0 : 0.0;
}

__global__ void add_diag_kernel(double* __restrict__ A, int64_t n, double alpha) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    A[i * n + i] += alpha;
}

template <typename T>
__global__ void check_finite_kernel(const T* __restrict__ x, int64_t n, int* __restrict__ flag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(static_cast<double>(x[i]));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

int grid_for(int64_t n, int threads = 256, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace {
int64_t gram_kchunk(int64_t K, int pairs, int64_t& chunks) {
  int64_t want = (4 * 152 + pairs - 1) / pairs;
  chunks = (K + 255) / 256;
  if (chunks > want) chunks = want;
  if (chunks < 1) chunks = 1;
  int64_t kchunk = (K + chunks - 1) / chunks;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  chunks = (K + kchunk - 1) / kchunk;
  return kchunk;
}
}  // namespace

template <typename T, typename Acc>
cudaError_t launch_gram(const T* X, double* G, int64_t A, int64_t I, int64_t B, cudaStream_t s) {
  if (A <= 0 || I <= 0 || B <= 0) return cudaSuccess;
  const int ntiles = (int)((I + TILE - 1) / TILE);
  const int pairs = ntiles * (ntiles + 1) / 2;
  const int64_t K = A * B;
  int64_t chunks = 1;
  const int64_t kchunk = gram_kchunk(K, pairs, chunks);
  dim3 grid(pairs, (unsigned)chunks);
  ProfScope prof(sizeof(Acc) == 8 ? K_GRAM_F64 : K_GRAM_F32, s, (double)I * (double)(I + 1) * (double)K,
                 (double)sizeof(T) * (double)K * (double)I + 8.0 * (double)I * (double)I);
  gram_simt_kernel<T, Acc><<<grid, NT, 0, s>>>(X, G, A, I, B, kchunk, ntiles);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_f64(const T* X, double* G, int64_t A, int64_t I, int64_t B, cudaStream_t s) {
  return launch_gram<T, double>(X, G, A, I, B, s);
}

cudaError_t launch_gram_f32(const float* X, double* G, int64_t A, int64_t I, int64_t B, cudaStream_t s) {
  if (I <= 64 && A * B >= 4 * CHC) {
    // short index: the streaming kernel (the caller zeroed G)
    const int Ip = (int)((I + 3) & ~3);
    const int T4 = Ip / 4, ntiles = T4 * (T4 + 1) / 2;
    const size_t sm = std::max(sizeof(float) * 2 * CHC * Ip, sizeof(double) * 16 * (size_t)ntiles);
    int64_t nb = (B == 1) ? 1 : (B >= CHC ? CHC : B), na = (B == 1) ? CHC : (B >= CHC ? 1 : CHC / B);
    const int64_t nchunks = ((A + na - 1) / na) * ((B == 1) ? 1 : (B + nb - 1) / nb);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(gram_small_kernel));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gram_small_kernel, GRAM_SMALL_THREADS, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<int64_t>(nchunks, (int64_t)std::min(per_sm, 4) * nsm);
    const int64_t K = A * B;
    ProfScope prof(K_GRAM_F32, s, (double)I * (double)(I + 1) * (double)K,
                   4.0 * (double)K * (double)I + 8.0 * (double)I * (double)I);
    gram_small_kernel<<<grid, GRAM_SMALL_THREADS, sm, s>>>(X, A, (int)I, B, G);
    note_launch();
    return cudaGetLastError();
  }
  return launch_gram<float, float>(X, G, A, I, B, s);
}

template <typename Tin, typename Tout, typename Acc, typename Tm>
cudaError_t launch_ttm(const Tin* X, Tout* out, const Tm* M, int64_t ms, int64_t mt, int64_t A, int64_t T,
                       int64_t B, int64_t S, int64_t R2, cudaStream_t s, int64_t S_store = -1,
                       double* resid = nullptr) {
  if (S_store < 0) S_store = S;
  if (A <= 0 || B <= 0 || S <= 0) return cudaSuccess;
  if (R2 < 1 || (B == 1 && A % R2 != 0) || (B > 1 && R2 != 1)) return cudaErrorInvalidValue;
  const int64_t AB = A * B;
  dim3 grid((unsigned)((AB + TILE - 1) / TILE), (unsigned)((S + TILE - 1) / TILE));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  ProfScope prof(sizeof(Acc) == 8 ? K_TTM_F64 : K_TTM_F32, s, 2.0 * (double)S * (double)T * (double)AB,
                 (double)sizeof(Tin) * (double)AB * (double)T + (double)sizeof(Tout) * (double)AB * (double)S);
  ttm_simt_kernel<Tin, Tout, Acc, Tm><<<grid, NT, 0, s>>>(X, out, M, ms, mt, A, T, B, S, R2, S_store, resid);
  note_launch();
  return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_ttm_f64(const Tin* X, Tout* out, const double* M, int64_t ms, int64_t mt, int64_t A,
                           int64_t T, int64_t B, int64_t S, cudaStream_t s) {
  return launch_ttm<Tin, Tout, double>(X, out, M, ms, mt, A, T, B, S, 1, s);
}

template <typename Tin>
cudaError_t launch_ttm_f32(const Tin* X, float* out, const float* M, int64_t ms, int64_t mt, int64_t A, int64_t T,
                           int64_t B, int64_t S, int64_t R2, cudaStream_t s) {
  return launch_ttm<Tin, float, float>(X, out, M, ms, mt, A, T, B, S, R2, s);
}

template <typename Tin>
cudaError_t launch_ttm_f32_resid(const Tin* X, float* out, const float* M, int64_t ms, int64_t mt, int64_t A,
                                 int64_t T, int64_t B, int64_t S, int64_t S_store, int64_t R2, double* resid,
                                 cudaStream_t s) {
  return launch_ttm<Tin, float, float>(X, out, M, ms, mt, A, T, B, S, R2, s, S_store, resid);
}

template <typename T>
cudaError_t launch_sqnorm(const T* x, int64_t n, double* acc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_NORM, s, 2.0 * (double)n, (double)sizeof(T) * (double)n);
  if constexpr (sizeof(T) == 4)
    sqnorm_f32_kernel<<<grid_for((n + 3) / 4, 256, 152 * 8), 256, 0, s>>>(x, n, acc);
  else
    sqnorm_kernel<T><<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(x, n, acc);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_trace(const double* G, int64_t n, double* acc, cudaStream_t s) {
  ProfScope prof(K_NORM, s);
  trace_kernel<<<1, 256, 0, s>>>(G, n, acc);
  note_launch();
  return cudaGetLastError();
}

template <int TE>
cudaError_t launch_gemm_tiles(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t a_rs,
                              int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs, double beta, double* C,
                              int64_t c_rs, int64_t c_cs, int nsm, cudaStream_t s) {
  const int64_t gx = (N + TE - 1) / TE, gy = (M + TE - 1) / TE;
  int64_t splits = 1, kchunk = std::max<int64_t>(K, 1);
  if (gx * gy < 4 * (int64_t)nsm && K > 2 * BK) {
    splits = std::min<int64_t>((4 * nsm + gx * gy - 1) / (gx * gy), (K + 2 * BK - 1) / (2 * BK));
    kchunk = ((K + splits - 1) / splits + BK - 1) / BK * BK;
    splits = (K + kchunk - 1) / kchunk;
  }
  if (splits > 1) {
    scale_strided_kernel<<<grid_for(M * N), 256, 0, s>>>(C, M, N, c_rs, c_cs, beta);
    note_launch();
  }
  gemm_f64_kernel<TE><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)splits), NT, 0, s>>>(
      M, N, K, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, C, c_rs, c_cs, kchunk);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t a_rs,
                            int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs, double beta, double* C,
                            int64_t c_rs, int64_t c_cs, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  ProfScope prof(K_GEMM_F64, s, 2.0 * (double)M * (double)N * (double)K,
                 8.0 * ((double)M * (double)K + (double)K * (double)N + (double)M * (double)N));
  if (N == 1 || M == 1) {
    // matrix-vector product: C(m, 0) = alpha A(m, :) B(:, 0) + beta C(m, 0), or its transpose for M == 1
    const bool col = (N == 1);
    const int64_t rows = col ? M : N;
    const int blocks = (int)std::min<int64_t>((rows + 7) / 8, 152 * 8);
    if (col)
      gemv_f64_kernel<<<blocks, 256, 0, s>>>(M, K, alpha, A, a_rs, a_cs, B, b_rs, beta, C, c_rs);
    else
      gemv_f64_kernel<<<blocks, 256, 0, s>>>(N, K, alpha, B, b_cs, b_rs, A, a_cs, beta, C, c_cs);
    note_launch();
    return cudaGetLastError();
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t mn = std::min(M, N);
  if (mn >= 256) return launch_gemm_tiles<64>(M, N, K, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, C, c_rs, c_cs, nsm, s);
  if (mn >= 48) return launch_gemm_tiles<32>(M, N, K, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, C, c_rs, c_cs, nsm, s);
  return launch_gemm_tiles<16>(M, N, K, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, C, c_rs, c_cs, nsm, s);
}

template <typename Tin, typename Tout>
cudaError_t launch_copy_pad3(const Tin* in, int64_t A1, int64_t B1, int64_t C1, Tout* out, int64_t A2,
                             int64_t B2, int64_t C2, cudaStream_t s) {
  const int64_t total = A2 * B2 * C2;
  if (total <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s, 0.0, (double)(sizeof(Tin) * A1 * B1 * C1 + sizeof(Tout) * total));
  copy_pad3_kernel<Tin, Tout><<<grid_for(total), 256, 0, s>>>(in, A1, B1, C1, out, A2, B2, C2);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_copy_cols(const double* in, int64_t ld_in, int64_t rows, int64_t cols, double* out,
                             int64_t ld_out, cudaStream_t s) {
  if (rows * cols <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  copy_cols_kernel<<<grid_for(rows * cols), 256, 0, s>>>(in, ld_in, rows, cols, out, ld_out);
  note_launch();
  return cudaGetLastError();
}

template <typename Tin, typename Tout>
cudaError_t launch_cast(const Tin* in, Tout* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  if (sizeof(Tin) == 4 && sizeof(Tout) == 8 && n % 4 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    cast_f32_f64_vec_kernel<<<grid_for(n / 4), 256, 0, s>>>(reinterpret_cast<const float4*>(in),
                                                             reinterpret_cast<double2*>(out), n / 4);
    note_launch();
    return cudaGetLastError();
  }
  cast_kernel<Tin, Tout><<<grid_for(n), 256, 0, s>>>(in, out, n);
  note_launch();
  return cudaGetLastError();
}

// out[c][r] = in[r][c] for a row-major [rows][cols] matrix: 32 x 32 tiles through shared memory so
// that both the reads and the writes are coalesced (the padding column avoids bank conflicts).
template <typename T>
__global__ void transpose2d_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t rows, int64_t cols) {
  __shared__ T tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += 8) {
    const int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][j];
  }
}

// out[a][b][t] = in[a][t][b] for t < T and 0 for T <= t < Tp: the middle axis of [A][T][B] moved innermost
// and padded (the tensor-core mode product reads rows of a multiple of four floats). 32 x 32 tiles
// through shared memory, batches over blockIdx.z.
__global__ void transpose_pad_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t A, int64_t T,
                                     int64_t B, int64_t Tp) {
  __shared__ float tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32, b0 = (int64_t)blockIdx.y * 32;
  for (int64_t a = blockIdx.z; a < A; a += gridDim.z) {
    const float* src = in + a * T * B;
    float* dst = out + a * B * Tp;
    for (int j = threadIdx.y; j < 32; j += 8) {
      const int64_t t = t0 + j, b = b0 + threadIdx.x;
      tile[j][threadIdx.x] = (t < T && b < B) ? src[t * B + b] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
      const int64_t b = b0 + j, t = t0 + threadIdx.x;
      if (b < B && t < Tp) dst[b * Tp + t] = tile[threadIdx.x][j];
    }
    __syncthreads();
  }
}

cudaError_t launch_transpose_pad(const float* in, float* out, int64_t A, int64_t T, int64_t B, int64_t Tp,
                                 cudaStream_t s) {
  if (A <= 0 || T <= 0 || B <= 0) return cudaSuccess;
  if (Tp < T) return cudaErrorInvalidValue;
  const int64_t gx = (Tp + 31) / 32, gy = (B + 31) / 32;
  if (gx > 2147483647LL || gy > 65535) return cudaErrorInvalidValue;
  ProfScope prof(K_COPY, s, 0.0, 4.0 * (double)A * (double)B * (double)(T + Tp));
  const dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)std::min<int64_t>(A, 65535)), block(32, 8);
  transpose_pad_kernel<<<grid, block, 0, s>>>(in, out, A, T, B, Tp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_transpose2d(const void* in, void* out, int64_t rows, int64_t cols, int elem_bytes,
                               cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int64_t gx = (cols + 31) / 32, gy = (rows + 31) / 32;
  if (gy > 65535 || gx > 2147483647LL || (elem_bytes != 4 && elem_bytes != 8)) return cudaErrorInvalidValue;
  ProfScope prof(K_COPY, s);
  const dim3 grid((unsigned)gx, (unsigned)gy), block(32, 8);
  if (elem_bytes == 4)
    transpose2d_kernel<float><<<grid, block, 0, s>>>(static_cast<const float*>(in), static_cast<float*>(out), rows,
                                                     cols);
  else
    transpose2d_kernel<double><<<grid, block, 0, s>>>(static_cast<const double*>(in), static_cast<double*>(out),
                                                      rows, cols);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale_cols_invsqrt(double* W, int64_t rows, int64_t cols, const double* lam, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  scale_cols_invsqrt_kernel<<<grid_for(rows * cols), 256, 0, s>>>(W, rows, cols, lam);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_uniform(double* X, int64_t n, uint64_t seed, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  fill_uniform_kernel<<<grid_for(n), 256, 0, s>>>(X, n, seed);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_unit_cols(double* Q, int64_t ldq, int64_t col0, int64_t ra0, int64_t rb0, int64_t ra, int64_t rb,
                             cudaStream_t s) {
  if (ra * rb <= ra0 * rb0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  unit_cols_kernel<<<grid_for(ra * rb), 256, 0, s>>>(Q, ldq, col0, ra0, rb0, ra, rb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_cast_matrix(const double* U, int64_t ms, int64_t mt, int64_t S, int64_t T, float* out,
                               cudaStream_t s) {
  if (S <= 0 || T <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  cast_matrix_kernel<<<grid_for(S * T), 256, 0, s>>>(U, ms, mt, S, T, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_identity(double* A, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  fill_identity_kernel<<<grid_for(n * n), 256, 0, s>>>(A, n);
  note_launch();
  return cudaGetLastError();
}


cudaError_t launch_add_diag(double* A, int64_t n, double alpha, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_COPY, s);
  add_diag_kernel<<<grid_for(n), 256, 0, s>>>(A, n, alpha);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(const T* x, int64_t n, int* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ProfScope prof(K_NORM, s);
  check_finite_kernel<T><<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(x, n, flag);
  note_launch();
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t launch_gram_f64<float>(const float*, double*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_gram_f64<double>(const double*, double*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f64<float, double>(const float*, double*, const double*, int64_t, int64_t, int64_t,
                                                   int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f64<double, double>(const double*, double*, const double*, int64_t, int64_t,
                                                    int64_t, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f64<float, float>(const float*, float*, const double*, int64_t, int64_t, int64_t,
                                                  int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f64<double, float>(const double*, float*, const double*, int64_t, int64_t,
                                                   int64_t, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_sqnorm<float>(const float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_sqnorm<double>(const double*, int64_t, double*, cudaStream_t);
template cudaError_t launch_copy_pad3<double, double>(const double*, int64_t, int64_t, int64_t, double*, int64_t,
                                                      int64_t, int64_t, cudaStream_t);
template cudaError_t launch_copy_pad3<float, float>(const float*, int64_t, int64_t, int64_t, float*, int64_t,
                                                    int64_t, int64_t, cudaStream_t);
template cudaError_t launch_copy_pad3<double, float>(const double*, int64_t, int64_t, int64_t, float*, int64_t,
                                                     int64_t, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f32<float>(const float*, float*, const float*, int64_t, int64_t, int64_t, int64_t,
                                           int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_ttm_f32_resid<float>(const float*, float*, const float*, int64_t, int64_t, int64_t,
                                                 int64_t, int64_t, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_ttm_f32_resid<double>(const double*, float*, const float*, int64_t, int64_t, int64_t,
                                                  int64_t, int64_t, int64_t, int64_t, int64_t, double*, cudaStream_t);
template cudaError_t launch_ttm_f32<double>(const double*, float*, const float*, int64_t, int64_t, int64_t, int64_t,
                                            int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_check_finite<float>(const float*, int64_t, int*, cudaStream_t);
template cudaError_t launch_check_finite<double>(const double*, int64_t, int*, cudaStream_t);

}  // namespace bht

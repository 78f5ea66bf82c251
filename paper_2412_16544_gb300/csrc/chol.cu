// chol.cu — certificate that every eigenvalue of a symmetric FP64 matrix G exceeds a bound tau: the
// Cholesky factorisation of G - sigma I, sigma = tau + delta, run in FP64 over 16 x 16 tiles across a
// cooperative grid.
//
// Use: the truncation of eq. ht_leaf_svd keeps every direction of a node exactly when the smallest
// eigenvalue of its Gram matrix exceeds the node's budget (the tail rule: the energy discarded by keeping
// n - 1 directions is the smallest eigenvalue). A factorisation that runs to completion decides such a
// node in about 2 n / 16 grid barriers and n^3 / 6 FMAs instead of its eigensolve.
//
// Rounding (Cholesky backward error, |dM| <= gamma_{n+1} |L||L^T| for the computed factor, as in
// Higham, Accuracy and Stability of Numerical Algorithms, Thm 10.3): a factorisation of
// M = fl(G - sigma I) that completes has L L^T = M + dM positive definite and
// ||dM||_2 <= ||dM||_F <= gamma_{n+1} ||L||_F^2 <= gamma_{n+1} trace(M) / (1 - gamma_{n+1}), so
// lambda_min(G) > sigma - ((n + 1) u (1 + O(n u)) + 2 u) trace(G). delta = 2 (n + 4) u trace(G), u = 2^-53,
// with the trace as computed, covers this with room for the rounding of the trace and of sigma itself
// (and for the pivots' reciprocal square roots, within one ulp, taken in place of a square root and
// divisions: a few more roundings per entry of L).
// A pivot <= 0 (or not a number) stops the factorisation: then no certificate is given.
#include <cmath>
#include <cstdint>

#include "internal.cuh"
#include "sync.cuh"

namespace bht {
namespace {

constexpr int PT = 16;               // tile edge
constexpr int PT_THREADS = PT * PT;  // one thread per entry of a tile

// (i, j), 0 <= j <= i, of the t-th lower-triangle tile in row order (t = i (i + 1) / 2 + j)
__device__ __forceinline__ void lower_tile(int t, int& i, int& j) {
  int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  i = r;
  j = t - r * (r + 1) / 2;
}

// A: n x n row-major workspace (lower tiles of G - sigma I, overwritten by the factor's tiles).
// fail: zero at launch; 1 + the step whose diagonal tile met a pivot <= 0. verdict: zero at launch, 1
// written at the end when the factorisation completed. Every step: the CTAs of the panel factor the
// diagonal tile (each its own copy, the same operations on the same values) and solve their panel tile
// against it; barrier; the failure word is read by every CTA (written only before this barrier, so every
// CTA reads the same value); the trailing tiles are updated; barrier.
__global__ void __launch_bounds__(PT_THREADS) spd_test_kernel(const double* __restrict__ G, int n, double tau,
                                                              double* __restrict__ A, Barrier* bar, int* fail,
                                                              int* verdict, int* status) {
  __shared__ double D[PT][PT + 1];  // diagonal tile; its strictly lower part becomes L_kk
  __shared__ double P[PT][PT + 1];  // panel tile (phase 1), row block i of the panel (phase 2)
  __shared__ double R[PT][PT + 1];  // row block j of the panel (phase 2)
  __shared__ double Li[PT];          // reciprocals of the diagonal of L_kk
  __shared__ int bad;
  __shared__ double red[33];
  const int tr = threadIdx.x / PT, tc = threadIdx.x % PT;
  unsigned int epoch = 0;

  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += G[(size_t)i * n + i];
  t = block_sum(t, red);  // the same value in every CTA
  const double sigma = tau + 2.0 * (double)(n + 4) * 0x1p-53 * t;
  if (!(t > 0.0) || !(sigma < INFINITY)) return;  // no certificate; the same decision in every CTA

  const int nblk = (n + PT - 1) / PT;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    if (i / PT >= j / PT) A[e] = (i == j) ? G[e] - sigma : G[e];
  }
  if (!grid_barrier_count(bar, epoch, status)) return;

  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * PT, kw = min(PT, n - k0);
    const int m = nblk - 1 - kb;  // tiles of the panel below the diagonal
    for (int c = blockIdx.x; c <= m; c += gridDim.x) {
      const int i0 = (kb + c) * PT, iw = min(PT, n - i0);
      D[tr][tc] = (tr < kw && tc <= tr) ? A[(size_t)(k0 + tr) * n + k0 + tc] : 0.0;
      if (c > 0) P[tr][tc] = (tr < iw && tc < kw) ? A[(size_t)(i0 + tr) * n + k0 + tc] : 0.0;
      __syncthreads();
      if (threadIdx.x == 0) {
        const double d = D[0][0];
        bad = !(d > 0.0);
        if (!bad) Li[0] = rsqrt(d);
      }
      __syncthreads();
      // Column j of the diagonal tile and of the panel tile (X L_kk^T = P) in two phases: the column
      // scaled by 1/L_jj; then the trailing updates, while thread 0 updates the next pivot and takes its
      // reciprocal square root, so that its scalar chain overlaps the other threads' updates.
      bool ok = true;
      for (int j = 0; j < kw; ++j) {
        if (bad) {  // written by thread 0 before the last barrier: the branch is uniform
          ok = false;
          break;
        }
        const double li = Li[j];
        if (tc == j && tr > j && tr < kw) D[tr][j] *= li;
        if (c > 0 && tc == j && tr < iw) P[tr][j] *= li;
        __syncthreads();
        if (tc > j && tr >= tc && tr < kw && !(tr == j + 1 && tc == j + 1)) D[tr][tc] -= D[tr][j] * D[tc][j];
        if (c > 0 && tc > j && tc < kw && tr < iw) P[tr][tc] -= P[tr][j] * D[tc][j];
        if (threadIdx.x == 0 && j + 1 < kw) {
          const double dn = D[j + 1][j + 1] - D[j + 1][j] * D[j + 1][j];
          D[j + 1][j + 1] = dn;
          bad = !(dn > 0.0);
          if (!bad) Li[j + 1] = rsqrt(dn);
        }
        __syncthreads();
      }
      if (!ok) {
        if (c == 0 && threadIdx.x == 0) atomicExch(fail, kb + 1);
        break;  // c is uniform in the CTA; a failed factor has nothing to solve against
      }
      if (c == 0) continue;
      if (tr < iw && tc < kw) A[(size_t)(i0 + tr) * n + k0 + tc] = P[tr][tc];
      __syncthreads();
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
    if (*(volatile int*)fail != 0) return;
    if (m == 0) break;
    // trailing update A_ij -= L_ik L_jk^T for kb < j <= i
    const int tiles = m * (m + 1) / 2;
    for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
      int bi, bj;
      lower_tile(tt, bi, bj);
      const int i0 = (kb + 1 + bi) * PT, j0 = (kb + 1 + bj) * PT;
      const int iw = min(PT, n - i0), jw = min(PT, n - j0);
      P[tr][tc] = (tr < iw && tc < kw) ? A[(size_t)(i0 + tr) * n + k0 + tc] : 0.0;
      R[tr][tc] = (tr < jw && tc < kw) ? A[(size_t)(j0 + tr) * n + k0 + tc] : 0.0;
      __syncthreads();
      if (tr < iw && tc < jw) {
        double* a = A + (size_t)(i0 + tr) * n + j0 + tc;
        double acc = *a;
#pragma unroll
        for (int k = 0; k < PT; ++k) acc -= P[tr][k] * R[tc][k];  // zero beyond kw
        *a = acc;
      }
      __syncthreads();
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *verdict = 1;
}

}  // namespace

size_t spd_test_workspace_bytes(int64_t n) {
  return ((sizeof(double) * (size_t)n * (size_t)n + 255) & ~(size_t)255) + 256;
}

cudaError_t launch_spd_test(const double* G, int64_t n, double tau, void* work, int* verdict, int* status,
                            cudaStream_t s) {
  if (n < 1 || n > 4096 || !(tau >= 0.0) || !std::isfinite(tau)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(work);
  double* A = reinterpret_cast<double*>(p);
  char* tail = p + ((sizeof(double) * (size_t)n * (size_t)n + 255) & ~(size_t)255);
  Barrier* bar = reinterpret_cast<Barrier*>(tail);
  int* fail = reinterpret_cast<int*>(tail + sizeof(Barrier));
  cudaError_t e = cudaMemsetAsync(tail, 0, sizeof(Barrier) + sizeof(int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(verdict, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int nblk = (int)((n + PT - 1) / PT);
  const int m0 = nblk - 1;
  int want = std::max(1, std::max(m0 + 1, m0 * (m0 + 1) / 2));
  const double nn = (double)n;
  ProfScope prof(K_SPD, s, nn * nn * nn / 3.0, 8.0 * nn * nn * 2.0);
  int ni = (int)n;
  if (want == 1) {
    spd_test_kernel<<<1, PT_THREADS, 0, s>>>(G, ni, tau, A, bar, fail, verdict, status);
    note_launch();
    return cudaGetLastError();
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spd_test_kernel, PT_THREADS, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one CTA per SM: more CTAs would only lengthen every grid barrier
  const int cap = nsm;
  const int grid = std::min(want, cap);
  void* args[] = {&G, &ni, &tau, &A, &bar, &fail, &verdict, &status};
  e = cudaLaunchCooperativeKernel((void*)spd_test_kernel, dim3(grid), dim3(PT_THREADS), args, 0, s);
  note_launch();
  return e;
}

}  // namespace bht

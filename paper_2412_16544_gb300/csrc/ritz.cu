// ritz.cu — eigenpairs of a small symmetric FP64 matrix (n <= 32) for the mixed-precision truncation of
// eq. ht_leaf_svd, in one CTA:
//   1. cyclic Jacobi in FP32 (round-robin ordering: n/2 disjoint rotations per round, applied to the rows,
//      then to the columns and to V), a rotation only where |a_pq| > 2^-23 sqrt(|a_pp a_qq|), until a sweep
//      rotates nothing or after 8 sweeps;
//   2. V to FP64, made orthonormal by two Newton-Schulz steps V <- V (3I - V^T V) / 2 (an orthonormality
//      error e becomes about 3e^2/4 per step);
//   3. the Ritz values h_i = v_i^T G v_i in FP64, sorted in decreasing order with their vectors.
// On GB300 the FP64 units issue at 1/64 of the FP32 rate, so the FP64 eigensolver's sequential chains
// (tridiagonalisation, bisection, inverse iteration) cost about 0.4 ms even at n = 24; here the iterative
// part runs in FP32 and FP64 only forms products.
//
// Why the truncation stays exact: with V orthonormal in FP64, keeping U = V[:, :r] discards exactly the
// energy trace(G) - sum_{i<r} h_i = sum_{i>=r} h_i of its own complement V[:, r:] (which becomes the node's
// orthonormal complement Q). The tail rule applied to the Ritz values therefore bounds the error of the
// basis actually kept, as eq. ht_leaf_svd requires. The Ritz values differ from the eigenvalues by the
// square of the FP32 vectors' angles (about 1e-14 of the matrix for separated eigenvalues), so the rank
// differs from the FP64 eigensolver's only when the tail meets eps_nw^2 within that.
#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace bht {
namespace {

constexpr int RZ_MAX = 32;
constexpr int RZ_THREADS = 256;
constexpr int RZ_SWEEPS = 8;

__global__ void __launch_bounds__(RZ_THREADS) small_ritz_kernel(const double* __restrict__ G, int n,
                                                                double* __restrict__ lam, double* __restrict__ Vout) {
  __shared__ float A[RZ_MAX][RZ_MAX + 1];
  __shared__ float V[RZ_MAX][RZ_MAX + 1];
  __shared__ float cs[RZ_MAX / 2][2];
  __shared__ int pq[RZ_MAX / 2][2];
  __shared__ double W[RZ_MAX][RZ_MAX + 1];   // FP64 V
  __shared__ double S[RZ_MAX][RZ_MAX + 1];   // V^T V, then G V
  __shared__ double Gs[RZ_MAX][RZ_MAX + 1];
  __shared__ double h[RZ_MAX];
  __shared__ double gmax[RZ_THREADS / 32];
  __shared__ int done;
  const int tid = threadIdx.x;
  const int m = n + (n & 1);  // an even number of players; index n (odd n) is a zero row and column
  double mx = 0.0;
  for (int e = tid; e < n * n; e += blockDim.x) {
    const double v = G[e];
    Gs[e / n][e % n] = v;
    mx = fmax(mx, fabs(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) gmax[tid >> 5] = mx;
  __syncthreads();
  mx = 0.0;
  for (int w = 0; w < RZ_THREADS / 32; ++w) mx = fmax(mx, gmax[w]);
  // the FP32 copy scaled by a power of two to a largest entry in [1, 2): no overflow in its squares
  int ex = 0;
  if (mx > 0.0 && mx < INFINITY) frexp(mx, &ex);
  for (int e = tid; e < RZ_MAX * RZ_MAX; e += blockDim.x) {
    const int i = e / RZ_MAX, j = e % RZ_MAX;
    A[i][j] = (i < n && j < n) ? (float)ldexp(Gs[i][j], 1 - ex) : 0.f;
    V[i][j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();

  // 1. FP32 cyclic Jacobi. A rotation is skipped when |a_pq| <= 2^-23 sqrt(|a_pp a_qq|) (the relative
  // criterion that keeps graded matrices accurate); the sweeps end when one skipped them all.
  for (int sweep = 0; sweep < RZ_SWEEPS; ++sweep) {
    if (tid == 0) done = 1;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      // pairs of this round (circle method: player m-1 fixed, the others rotate)
      if (tid < m / 2) {
        int p, q;
        if (tid == 0) {
          p = round;
          q = m - 1;
        } else {
          p = (round + tid) % (m - 1);
          q = (round - tid + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        float c = 1.f, sn = 0.f;
        const float apq = A[p][q];
        if (q < n && apq != 0.f && fabsf(apq) > 0x1p-23f * sqrtf(fabsf(A[p][p] * A[q][q]))) {
          done = 0;
          const float tau = (A[q][q] - A[p][p]) / (2.f * apq);
          const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = 1.f / sqrtf(1.f + t * t);
          sn = t * c;
        }
        pq[tid][0] = p;
        pq[tid][1] = q;
        cs[tid][0] = c;
        cs[tid][1] = sn;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < (m / 2) * m; e += blockDim.x) {
        const int k = e / m, j = e % m;
        const int p = pq[k][0], q = pq[k][1];
        const float c = cs[k][0], sn = cs[k][1];
        const float ap = A[p][j], aq = A[q][j];
        A[p][j] = c * ap - sn * aq;
        A[q][j] = sn * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < (m / 2) * m; e += blockDim.x) {
        const int k = e / m, i = e % m;
        const int p = pq[k][0], q = pq[k][1];
        const float c = cs[k][0], sn = cs[k][1];
        const float ap = A[i][p], aq = A[i][q];
        A[i][p] = c * ap - sn * aq;
        A[i][q] = sn * ap + c * aq;
        const float vp = V[i][p], vq = V[i][q];
        V[i][p] = c * vp - sn * vq;
        V[i][q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
    const int stop = done;  // read after the round's last barrier: the same value in every thread
    __syncthreads();        // ... before thread 0 resets it for the next sweep
    if (stop) break;
  }

  // 2. FP64 V, two Newton-Schulz steps
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    W[i][j] = (double)V[i][j];
  }
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    for (int e = tid; e < n * n; e += blockDim.x) {  // S = V^T V
      const int i = e / n, j = e % n;
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(W[k][i], W[k][j], acc);
      S[i][j] = acc;
    }
    __syncthreads();
    double nv[4];
    int cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) {  // V (3I - S) / 2, at most four entries a thread
      const int i = e / n, j = e % n;
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc = fma(W[i][k], (k == j ? 3.0 : 0.0) - S[k][j], acc);
      nv[cnt] = 0.5 * acc;
    }
    __syncthreads();
    cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) W[e / n][e % n] = nv[cnt];
    __syncthreads();
  }
  // 3. Ritz values: S = G V, h_j = v_j^T (G v_j)
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(Gs[i][k], W[k][j], acc);
    S[i][j] = acc;
  }
  __syncthreads();
  if (tid < n) {
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(W[k][tid], S[k][tid], acc);
    h[tid] = acc;
  }
  __syncthreads();
  // sorted decreasing (ties by index): column j goes to its rank
  if (tid < n) {
    const double hj = h[tid];
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += (h[k] > hj || (h[k] == hj && k < tid)) ? 1 : 0;
    lam[rank] = hj;
    for (int i = 0; i < n; ++i) Vout[i * n + rank] = W[i][tid];
  }
}

}  // namespace

cudaError_t launch_small_ritz(const double* G, int64_t n, double* lam, double* V, cudaStream_t s) {
  if (n < 1 || n > RZ_MAX) return cudaErrorInvalidValue;
  ProfScope prof(K_RITZ, s, 4.0 * (double)n * n * n * 8.0, 8.0 * (double)n * n * 2.0);
  small_ritz_kernel<<<1, RZ_THREADS, 0, s>>>(G, (int)n, lam, V);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

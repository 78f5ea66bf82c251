// ritz.cu — eigenpairs of a small symmetric FP64 matrix (n <= 32) for the mixed-precision truncation of
// eq. ht_leaf_svd, in one CTA:
//   1. cyclic Jacobi in FP32 (round-robin ordering: n/2 disjoint rotations per round, applied as 2 x 2
//      blocks of J^T A J and columns of V J), a rotation only where |a_pq| > 2^-23 sqrt(|a_pp a_qq|), until a
//      sweep rotates nothing or after 8 sweeps;
//   2. V to FP64, made orthonormal by two Newton-Schulz steps V <- V (3I - V^T V) / 2 (an orthonormality
//      error e becomes about 3e^2/4 per step);
//   3. one FP64 refinement of the vectors (first-order eigenvectors of V^T G V, then Newton-Schulz);
//   4. the Ritz values h_i = v_i^T G v_i in FP64, sorted in decreasing order with their vectors.
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
  __shared__ float4 rot[RZ_MAX / 2];  // (p, q as bits, c, s) of the round's rotations
  __shared__ int done;
  __shared__ double W[RZ_MAX][RZ_MAX + 1];   // FP64 V
  __shared__ double S[RZ_MAX][RZ_MAX + 1];   // V^T V, then G V
  __shared__ double Gs[RZ_MAX][RZ_MAX + 1];
  __shared__ double Hm[RZ_MAX][RZ_MAX + 1];  // V^T G V in the refinement
  __shared__ double h[RZ_MAX];
  __shared__ double gmax[RZ_THREADS / 32];
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
  // criterion that keeps graded matrices accurate); the sweeps end when one skipped them all. A round
  // applies its m/2 disjoint rotations in one phase: thread (x, y) owns the 2 x 2 block of rows of pair x
  // and columns of pair y and forms (J^T A J) there from the old entries; the columns of V likewise. The
  // tasks of a thread are the same in every round, so their indices are taken once.
  const int hp = m / 2;
  const bool blk = tid < hp * hp;
  const int kx = blk ? tid / hp : 0, ky = blk ? tid - (tid / hp) * hp : 0;
  int vi[2], vk[2];
  for (int u = 0; u < 2; ++u) {
    const int e = tid + u * RZ_THREADS;
    vi[u] = e < m * hp ? e / hp : -1;
    vk[u] = e < m * hp ? e - (e / hp) * hp : 0;
  }
  for (int sweep = 0; sweep < RZ_SWEEPS; ++sweep) {
    if (tid == 0) done = 1;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      // pairs of this round (circle method: player m-1 fixed, the others rotate)
      if (tid < hp) {
        int p = round, q = m - 1;
        if (tid > 0) {
          p = round + tid;
          if (p >= m - 1) p -= m - 1;
          q = round - tid;
          if (q < 0) q += m - 1;
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
          const float tau = __fdividef(A[q][q] - A[p][p], 2.f * apq);
          float t;
          if (fabsf(tau) > 1e15f) {
            t = __fdividef(0.5f, tau);
          } else {
            const float hh = 1.f + tau * tau;
            t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + hh * rsqrtf(hh));
          }
          c = rsqrtf(1.f + t * t);
          sn = t * c;
        }
        rot[tid] = make_float4(__int_as_float(p), __int_as_float(q), c, sn);
      }
      __syncthreads();
      if (blk) {
        const float4 rx = rot[kx], ry = rot[ky];
        const int px = __float_as_int(rx.x), qx = __float_as_int(rx.y);
        const int py = __float_as_int(ry.x), qy = __float_as_int(ry.y);
        const float cx = rx.z, sx = rx.w, cy = ry.z, sy = ry.w;
        const float a = A[px][py], b = A[px][qy], c = A[qx][py], d = A[qx][qy];
        const float rp0 = cx * a - sx * c, rp1 = cx * b - sx * d;  // row p of J^T A
        const float rq0 = sx * a + cx * c, rq1 = sx * b + cx * d;  // row q
        A[px][py] = cy * rp0 - sy * rp1;
        A[px][qy] = sy * rp0 + cy * rp1;
        A[qx][py] = cy * rq0 - sy * rq1;
        A[qx][qy] = sy * rq0 + cy * rq1;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (vi[u] < 0) continue;
        const float4 ry = rot[vk[u]];
        const int py = __float_as_int(ry.x), qy = __float_as_int(ry.y);
        const float vp = V[vi[u]][py], vq = V[vi[u]][qy];
        V[vi[u]][py] = ry.z * vp - ry.w * vq;
        V[vi[u]][qy] = ry.w * vp + ry.z * vq;
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
  // products with four partial sums per entry: dependency chains a quarter as long
  auto dot4 = [&](const double* a, int sa, const double* b, int sb) {
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    int k = 0;
    for (; k + 4 <= n; k += 4) {
      c0 = fma(a[k * sa], b[k * sb], c0);
      c1 = fma(a[(k + 1) * sa], b[(k + 1) * sb], c1);
      c2 = fma(a[(k + 2) * sa], b[(k + 2) * sb], c2);
      c3 = fma(a[(k + 3) * sa], b[(k + 3) * sb], c3);
    }
    for (; k < n; ++k) c0 = fma(a[k * sa], b[k * sb], c0);
    return (c0 + c1) + (c2 + c3);
  };
  constexpr int LD = RZ_MAX + 1;
  for (int step = 0; step < 2; ++step) {
    for (int e = tid; e < n * n; e += blockDim.x) {  // S = (3I - V^T V) / 2
      const int i = e / n, j = e % n;
      S[i][j] = (i == j ? 1.5 : 0.0) - 0.5 * dot4(&W[0][i], LD, &W[0][j], LD);
    }
    __syncthreads();
    double nv[4];
    int cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) {  // V S, at most four entries a thread
      const int i = e / n, j = e % n;
      nv[cnt] = dot4(&W[i][0], 1, &S[0][j], LD);
    }
    __syncthreads();
    cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) W[e / n][e % n] = nv[cnt];
    __syncthreads();
  }
  // 2b. One FP64 refinement of the vectors. The FP32 vectors are eigenvectors of G rounded to FP32, so the
  // subspace they span is off by up to u32 ||G|| / gap (1e-5 .. 1e-4 rad for gaps of 1e-3 of the trace).
  // With H = V^T G V = D + E (E off the diagonal, of that size), the eigenvectors of H are I + Z to first
  // order, Z_ij = E_ij / (D_jj - D_ii): V (I + Z) leaves an error of order (E / gap)^2, and two
  // Newton-Schulz steps restore orthonormality (Z is antisymmetric). Pairs whose gap is below a thousand
  // times their coupling (a cluster) keep their vectors: rotations inside a cluster leave the split between
  // kept and discarded directions alone unless the split falls inside it, a tie either way.
  for (int e = tid; e < n * n; e += blockDim.x) {  // S = G V
    const int i = e / n, j = e % n;
    S[i][j] = dot4(&Gs[i][0], 1, &W[0][j], LD);
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {  // H = V^T S
    const int i = e / n, j = e % n;
    Hm[i][j] = dot4(&W[0][i], LD, &S[0][j], LD);
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += blockDim.x) {  // Z (into S), with I added: S = I + Z
    const int i = e / n, j = e % n;
    double z = (i == j) ? 1.0 : 0.0;
    if (i != j) {
      const double eij = 0.5 * (Hm[i][j] + Hm[j][i]), d = Hm[j][j] - Hm[i][i];
      if (d != 0.0 && fabs(eij) <= 1e-3 * fabs(d)) z = eij / d;
    }
    S[i][j] = z;
  }
  __syncthreads();
  {
    double nv[4];
    int cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) {  // V (I + Z)
      const int i = e / n, j = e % n;
      nv[cnt] = dot4(&W[i][0], 1, &S[0][j], LD);
    }
    __syncthreads();
    cnt = 0;
    for (int e = tid; e < n * n; e += blockDim.x, ++cnt) W[e / n][e % n] = nv[cnt];
    __syncthreads();
    for (int step = 0; step < 2; ++step) {
      for (int e = tid; e < n * n; e += blockDim.x) {  // S = (3I - V^T V) / 2
        const int i = e / n, j = e % n;
        S[i][j] = (i == j ? 1.5 : 0.0) - 0.5 * dot4(&W[0][i], LD, &W[0][j], LD);
      }
      __syncthreads();
      cnt = 0;
      for (int e = tid; e < n * n; e += blockDim.x, ++cnt) {  // V S
        const int i = e / n, j = e % n;
        nv[cnt] = dot4(&W[i][0], 1, &S[0][j], LD);
      }
      __syncthreads();
      cnt = 0;
      for (int e = tid; e < n * n; e += blockDim.x, ++cnt) W[e / n][e % n] = nv[cnt];
      __syncthreads();
    }
  }
  // 3. Ritz values: S = G V, h_j = v_j^T (G v_j)
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    S[i][j] = dot4(&Gs[i][0], 1, &W[0][j], LD);
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

// eig.cu — FP64 symmetric eigensolvers for the node truncations.
//
// The error-truncated SVD of a node unfolding (eq. ht_leaf_svd, eq.
// svd_on_residual) keeps the left singular vectors; they are the
// eigenvectors of the unfolding's Gram matrix, with eigenvalues sigma_i^2.
// Both solvers below run the cyclic Jacobi method with the round-robin
// (circle) ordering: every round rotates n/2 disjoint index pairs at once, and
// one round is written as independent 2 x 2 block updates
//     A[P_i, P_j] <- J_i^T A[P_i, P_j] J_j ,   P_i = {p_i, q_i},
// so a round needs one barrier, not two.
//   * eig_small: one CTA per matrix, A in shared memory (n <= 128).
//   * eig_coop : one cooperative grid, A in global memory (L2-resident), a
//                bounded grid barrier per round; every CTA recomputes the
//                round's rotations itself, so no rotation data is exchanged.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace bht {

namespace {

constexpr int SMALL_MAX = 128;
constexpr int EIG_THREADS = 256;
constexpr int MAX_SWEEPS = 40;
constexpr double EPS_REL = 2.220446049250313e-16;

struct Rot {
  double c, s;
};

// Pair k of round r among m = n2 - 1 rotating players (n2 even).
__device__ __forceinline__ void round_pair(int r, int k, int m, int& p, int& q) {
  if (k == 0) {
    p = r;
    q = m;
  } else {
    p = (r + k) % m;
    q = (r - k + m) % m;
  }
}

// Symmetric Schur 2x2: (c, s) zeroing a_pq of [[a_pp, a_pq], [a_pq, a_qq]].
__device__ __forceinline__ Rot schur2(double app, double aqq, double apq, double abs_tol, bool& rotated) {
  Rot r{1.0, 0.0};
  rotated = false;
  const double aa = fabs(apq);
  if (aa <= abs_tol || aa <= EPS_REL * sqrt(fabs(app) * fabs(aqq))) return r;
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  r.c = 1.0 / sqrt(1.0 + t * t);
  r.s = t * r.c;
  rotated = true;
  return r;
}

// 2x2 block update of A at rows (pi, qi), cols (pj, qj); `n` real size, indices
// >= n are the dummy player (zero row / column).
template <bool Symmetric>
__device__ __forceinline__ void block_update(double* A, int64_t lda, int n, int pi, int qi, Rot ri, int pj, int qj,
                                             Rot rj, bool diag) {
  const bool vi = qi < n, vj = qj < n;
  double m00 = A[(int64_t)pi * lda + pj];
  double m01 = vj ? A[(int64_t)pi * lda + qj] : 0.0;
  double m10 = vi ? A[(int64_t)qi * lda + pj] : 0.0;
  double m11 = (vi && vj) ? A[(int64_t)qi * lda + qj] : 0.0;
  // rows: J_i^T M
  const double r00 = ri.c * m00 - ri.s * m10, r01 = ri.c * m01 - ri.s * m11;
  const double r10 = ri.s * m00 + ri.c * m10, r11 = ri.s * m01 + ri.c * m11;
  // cols: (.) J_j
  double n00 = rj.c * r00 - rj.s * r01, n01 = rj.s * r00 + rj.c * r01;
  double n10 = rj.c * r10 - rj.s * r11, n11 = rj.s * r10 + rj.c * r11;
  if (diag) {  // the rotated pair itself: off-diagonal is zero by construction
    n01 = 0.0;
    n10 = 0.0;
  }
  A[(int64_t)pi * lda + pj] = n00;
  if (vj) A[(int64_t)pi * lda + qj] = n01;
  if (vi) A[(int64_t)qi * lda + pj] = n10;
  if (vi && vj) A[(int64_t)qi * lda + qj] = n11;
  if (Symmetric && !diag) {  // mirror into the lower half
    A[(int64_t)pj * lda + pi] = n00;
    if (vj) A[(int64_t)qj * lda + pi] = n01;
    if (vi) A[(int64_t)pj * lda + qi] = n10;
    if (vi && vj) A[(int64_t)qj * lda + qi] = n11;
  }
}

__device__ __forceinline__ void vt_update(double* VT, int n, int p, int q, Rot r, int k) {
  if (q >= n) return;
  const double a = VT[(int64_t)p * n + k], b = VT[(int64_t)q * n + k];
  VT[(int64_t)p * n + k] = r.c * a - r.s * b;
  VT[(int64_t)q * n + k] = r.s * a + r.c * b;
}

// ---------------------------------------------------------------------------
// small: one CTA per matrix, A in shared memory
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EIG_THREADS) eig_small_kernel(const double* __restrict__ G, int n,
                                                                double* __restrict__ lam, double* __restrict__ V,
                                                                double* __restrict__ VT) {
  extern __shared__ double smem[];
  const int n2 = n + (n & 1);
  const int m = n2 - 1;
  const int np = n2 / 2;
  double* A = smem;                          // n x n, lda = n
  Rot* rot = reinterpret_cast<Rot*>(A + (int64_t)n * n);  // np
  int* rank = reinterpret_cast<int*>(rot + np);           // n
  __shared__ int any_rot;
  __shared__ double normA;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    A[e] = G[e];
    const int i = e / n, k = e - i * n;
    VT[e] = (i == k) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int e = 0; e < n * n; ++e) s += A[e] * A[e];
    normA = sqrt(s);
  }
  __syncthreads();
  const double abs_tol = 1e-17 * normA;
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) any_rot = 0;
    __syncthreads();
    for (int r = 0; r < m; ++r) {
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int p, q;
        round_pair(r, k, m, p, q);
        bool did = false;
        Rot rr{1.0, 0.0};
        if (q < n) rr = schur2(A[p * n + p], A[q * n + q], A[p * n + q], abs_tol, did);
        rot[k] = rr;
        if (did) any_rot = 1;
      }
      __syncthreads();
      const int nblk = np * (np + 1) / 2;
      for (int w = threadIdx.x; w < nblk; w += blockDim.x) {
        int i = 0, rem = w;
        while (rem >= np - i) { rem -= np - i; ++i; }
        const int j = i + rem;
        int pi, qi, pj, qj;
        round_pair(r, i, m, pi, qi);
        round_pair(r, j, m, pj, qj);
        if (pi >= n) { int t = pi; pi = qi; qi = t; }
        if (pj >= n) { int t = pj; pj = qj; qj = t; }
        Rot ri = rot[i], rj = rot[j];
        block_update<true>(A, n, n, pi, qi, ri, pj, qj, rj, i == j);
      }
      for (int w = threadIdx.x; w < np * n; w += blockDim.x) {
        const int k = w / n, col = w - k * n;
        int p, q;
        round_pair(r, k, m, p, q);
        if (p >= n) continue;
        vt_update(VT, n, p, q, rot[k], col);
      }
      __syncthreads();
    }
    if (!any_rot) break;
    __syncthreads();
  }
  // sort eigenvalues descending (ties by index) and scatter eigenvectors
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = A[i * n + i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j * n + j];
      rk += (lj > li) || (lj == li && j < i);
    }
    rank[i] = rk;
    lam[rk] = li;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, k = e - i * n;  // eigenvector i, component k
    V[(int64_t)k * n + rank[i]] = VT[e];
  }
}

// ---------------------------------------------------------------------------
// cooperative: A in global memory, bounded grid barrier
// ---------------------------------------------------------------------------
struct Barrier {
  unsigned int count;
  unsigned int gen;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the wait gave up (status set to BHT_ETIMEOUT = 6).
__device__ bool grid_barrier(Barrier* bar, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*vgen == g) {
        if (*(volatile int*)status != 0) { ok = 0; break; }
        if (global_ns() - t0 > 1000000000ull) {  // 1 s
          atomicExch(status, 6);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Partner of index x in round r (m rotating players, dummy/fixed player m).
__device__ __forceinline__ int round_partner(int x, int r, int m) {
  if (x == m) return r;
  if (x == r) return m;
  int y = (2 * r - x) % m;
  return y < 0 ? y + m : y;
}

// Slot (0 .. np-1) of the pair containing index x in round r.
__device__ __forceinline__ int round_slot(int x, int r, int m) {
  if (x == m || x == r) return 0;
  int k = (x - r) % m;
  if (k < 0) k += m;
  return k < m - k ? k : m - k;
}

__global__ void __launch_bounds__(EIG_THREADS) eig_coop_kernel(double* __restrict__ A, int n,
                                                               double* __restrict__ lam, double* __restrict__ V,
                                                               double* __restrict__ VT, Barrier* bar,
                                                               int* status, double normA,
                                                               double* __restrict__ diagv,   // [2][n2]
                                                               double* __restrict__ offv) {  // [2][np]
  extern __shared__ double smem[];
  const int n2 = n + (n & 1);
  const int m = n2 - 1;
  const int np = n2 / 2;
  Rot* rot = reinterpret_cast<Rot*>(smem);        // np
  __shared__ int any_rot;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = gtid; e < (int64_t)n * n; e += gsz) {
    const int64_t i = e / n, k = e - i * n;
    VT[e] = (i == k) ? 1.0 : 0.0;
  }
  // snapshots read by the rotation computation of the first round
  for (int64_t x = gtid; x < n2; x += gsz) diagv[x] = (x < n) ? A[x * n + x] : 0.0;
  for (int64_t k = gtid; k < np; k += gsz) {
    int p, q;
    round_pair(0, (int)k, m, p, q);
    offv[k] = (p < n && q < n) ? A[(int64_t)p * n + q] : 0.0;
  }
  if (!grid_barrier(bar, status)) return;
  const double abs_tol = 1e-17 * normA;
  const int64_t nblk = (int64_t)np * (np + 1) / 2;
  int64_t gr = 0;  // rounds executed so far: selects the snapshot buffer
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) any_rot = 0;
    __syncthreads();
    for (int r = 0; r < m; ++r, ++gr) {
      const double* dcur = diagv + (gr & 1) * n2;
      const double* ocur = offv + (gr & 1) * np;
      double* dnext = diagv + ((gr + 1) & 1) * n2;
      double* onext = offv + ((gr + 1) & 1) * np;
      const int rn = (r + 1 == m) ? 0 : r + 1;  // next round (wraps into the next sweep)
      // every CTA derives the same rotations from the same snapshot values
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int p, q;
        round_pair(r, k, m, p, q);
        bool did = false;
        Rot rr{1.0, 0.0};
        if (q < n && p < n) rr = schur2(dcur[p], dcur[q], ocur[k], abs_tol, did);
        rot[k] = rr;
        if (did) any_rot = 1;
      }
      __syncthreads();
      // upper-triangular block pairs (i <= j); consecutive threads take consecutive j
      for (int64_t w = gtid; w < nblk; w += gsz) {
        const double b2 = 2.0 * np + 1.0;
        int i = (int)((b2 - sqrt(b2 * b2 - 8.0 * (double)w)) * 0.5);
        if (i < 0) i = 0;
        if (i > np - 1) i = np - 1;
        int64_t start = (int64_t)i * np - (int64_t)i * (i - 1) / 2;
        while (start > w) { --i; start = (int64_t)i * np - (int64_t)i * (i - 1) / 2; }
        while (start + (np - i) <= w) { start += np - i; ++i; }
        const int j = i + (int)(w - start);
        int pi, qi, pj, qj;
        round_pair(r, i, m, pi, qi);
        round_pair(r, j, m, pj, qj);
        block_update<true>(A, n, n, pi, qi, rot[i], pj, qj, rot[j], i == j);
        // publish what the next round's rotations read
        const int xs[2] = {pi, qi}, ys[2] = {pj, qj};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int x = xs[u], y = ys[v];
            if (x >= n || y >= n) continue;
            const double val = A[(int64_t)x * n + y];
            if (x == y) {
              dnext[x] = val;
            } else if (round_partner(x, rn, m) == y && (i != j || x < y)) {
              onext[round_slot(x, rn, m)] = val;
            }
          }
      }
      for (int64_t w = gtid; w < (int64_t)np * n; w += gsz) {
        const int k = (int)(w / n), col = (int)(w - (int64_t)k * n);
        int p, q;
        round_pair(r, k, m, p, q);
        if (p >= n) continue;
        vt_update(VT, n, p, q, rot[k], col);
      }
      if (!grid_barrier(bar, status)) return;
    }
    __syncthreads();
    if (!any_rot) break;
  }
  // every CTA ranks the eigenvalues itself and writes its share of V
  int* rank = reinterpret_cast<int*>(smem);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double li = A[(int64_t)i * n + i];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[(int64_t)j * n + j];
      rk += (lj > li) || (lj == li && j < i);
    }
    rank[i] = rk;
    if (blockIdx.x == 0) lam[rk] = li;
  }
  __syncthreads();
  for (int64_t e = gtid; e < (int64_t)n * n; e += gsz) {
    const int64_t i = e / n, k = e - i * n;
    V[k * n + rank[i]] = VT[e];
  }
}

__global__ void fro_norm_kernel(const double* __restrict__ A, int64_t nn, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(A[i], A[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

size_t small_smem_bytes(int64_t n) {
  const int64_t n2 = n + (n & 1);
  return (size_t)(n * n) * sizeof(double) + (size_t)(n2 / 2) * sizeof(Rot) + (size_t)n * sizeof(int) + 16;
}

}  // namespace

size_t eig_workspace_bytes(int64_t n) {
  // VT (n x n) + barrier + norm scalar + two rounds of rotation snapshots
  size_t vt = ((size_t)(n * n) * sizeof(double) + 255) & ~(size_t)255;
  size_t snap = ((size_t)(2 * (n + 1) + 2 * (n / 2 + 1)) * sizeof(double) + 255) & ~(size_t)255;
  return vt + 256 + 256 + snap;
}

cudaError_t launch_eig_sym(double* G, int64_t n, double* lam, double* V, void* work, int* status,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 8192) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(work);
  double* VT = reinterpret_cast<double*>(w);
  size_t vt = ((size_t)(n * n) * sizeof(double) + 255) & ~(size_t)255;
  Barrier* bar = reinterpret_cast<Barrier*>(w + vt);
  double* nrm = reinterpret_cast<double*>(w + vt + 256);
  const int64_t n2e = n + (n & 1);
  double* diagv = reinterpret_cast<double*>(w + vt + 512);
  double* offv = diagv + 2 * n2e;
  if (n <= SMALL_MAX) {
    const size_t sm = small_smem_bytes(n);
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(eig_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_set = true;
    }
    ProfScope prof(K_EIG_SMALL, s, 9.0 * (double)n * (double)n * (double)n, 24.0 * (double)n * (double)n);
    eig_small_kernel<<<1, EIG_THREADS, sm, s>>>(G, (int)n, lam, V, VT);
    note_launch();
    return cudaGetLastError();
  }
  // Frobenius norm for the absolute rotation threshold, read back to the host
  cudaError_t e = cudaMemsetAsync(nrm, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  {
    ProfScope prof(K_NORM, s);
    fro_norm_kernel<<<152, 256, 0, s>>>(G, n * n, nrm);
  }
  note_launch();
  double h_nrm = 0.0;
  e = cudaMemcpyAsync(&h_nrm, nrm, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  h_nrm = sqrt(h_nrm);
  e = cudaMemsetAsync(bar, 0, sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  int dev = 0;
  cudaGetDevice(&dev);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n2 = n + (n & 1);
  const size_t sm = (size_t)(n2 / 2) * sizeof(Rot) + 64;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(eig_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eig_coop_kernel, EIG_THREADS, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = nsm * (per_sm > 2 ? 2 : per_sm);
  int nn = (int)n;
  void* args[] = {&G, &nn, &lam, &V, &VT, &bar, &status, &h_nrm, &diagv, &offv};
  {
    ProfScope prof(K_EIG_COOP, s, 9.0 * (double)n * (double)n * (double)n, 24.0 * (double)n * (double)n);
    e = cudaLaunchCooperativeKernel((void*)eig_coop_kernel, dim3(blocks), dim3(EIG_THREADS), args, sm, s);
  }
  note_launch();
  return e;
}

}  // namespace bht

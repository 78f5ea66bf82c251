// wy.cu — a product of Householder reflectors applied to many vectors, in blocks.
//
// x <- H_0 H_1 ... H_{K-1} x for H_k = I - tau_k v_k v_k^T, where v_k is zero above row k + off and 1 at
// row k + off. Consecutive reflectors are grouped by the compact WY representation (Schreiber and Van
// Loan, 1989): H_{k0} H_{k0+1} ... H_{k0+kb-1} = I - V T V^T with V = [v_{k0} .. v_{k0+kb-1}] and T upper
// triangular, T_jj = tau_j and T(0:j, j) = -tau_j T(0:j, 0:j) V(:, 0:j)^T v_j. A block then costs two thin
// products, w = V^T x and x -= V (T w), for all of a CTA's vectors at once, instead of kb dependent
// chains of a dot product, a warp reduction and an update per vector. The FP64 work is the same; what
// goes is the latency of the chain, which left the one-warp-per-vector form far below the FP64 pipe's
// rate on every size this library meets.
//
// Two users: the back-transformation of a tridiagonal matrix's eigenvectors (reflector k acts on rows
// k + 1 .., stored from position 0 of row k of Vh), and the orthonormal complement from a Householder QR
// (reflector j acts on rows j .., stored at its absolute rows of row j of V), applied to the unit vectors
// e_k .. e_{c-1}. A reflector with tau = 0 is the identity; its stored entries are never read.
#include <algorithm>

#include "internal.cuh"
#include "sync.cuh"

namespace bht {

namespace {

constexpr int WY_THREADS = 256;
constexpr int WY_NB = 16;  // reflectors per block, at most

// Entry i (>= k + off) of v_k: V[k * ldv + i - rel * (k + off)].
__device__ __forceinline__ int64_t refl_index(int64_t ldv, int off, int rel, int k, int i) {
  return (int64_t)k * ldv + i - (int64_t)rel * (k + off);
}

// T of each block of nb reflectors (the last block may be shorter), [nblk][nb][nb] row-major, zero below
// the diagonal and outside the block. One CTA per block: the Gram entries S(p, l) = v_p^T v_l (p < l),
// one warp each, then the columns of T one after another on warp 0.
__global__ void __launch_bounds__(WY_THREADS) wy_tfactor_kernel(const double* __restrict__ V, int64_t ldv, int off,
                                                                int rel, const double* __restrict__ tau, int K,
                                                                int L, int nb, double* __restrict__ Tg) {
  __shared__ double S[WY_NB][WY_NB + 1];
  __shared__ double T[WY_NB][WY_NB + 1];
  const int b = blockIdx.x, k0 = b * nb, kb = min(nb, K - k0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = warp; q < kb * kb; q += nw) {
    const int p = q / kb, l = q - p * kb;
    if (p >= l) continue;
    const int kp = k0 + p, kl = k0 + l;
    double acc = 0.0;
    if (tau[kp] != 0.0 && tau[kl] != 0.0) {
      // v_l starts at row kl + off, below the start of v_p
      double part[4] = {0.0, 0.0, 0.0, 0.0};  // four loads of each vector in flight per lane
      int i = kl + off + lane;
      for (; i + 96 < L; i += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          part[u] = fma(V[refl_index(ldv, off, rel, kp, i + 32 * u)], V[refl_index(ldv, off, rel, kl, i + 32 * u)],
                        part[u]);
      }
      for (; i < L; i += 32)
        part[0] = fma(V[refl_index(ldv, off, rel, kp, i)], V[refl_index(ldv, off, rel, kl, i)], part[0]);
      acc = warp_sum((part[0] + part[1]) + (part[2] + part[3]));
    }
    if (lane == 0) S[p][l] = acc;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < kb; ++j) {
      const double tj = tau[k0 + j];
      if (lane < j) {  // T(lane, j) = -tau_j sum_{lane <= p < j} T(lane, p) S(p, j)
        double acc = 0.0;
        for (int p = lane; p < j; ++p) acc = fma(T[lane][p], S[p][j], acc);
        T[lane][j] = -tj * acc;
      } else if (lane == j) {
        T[j][j] = tj;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    Tg[(int64_t)b * nb * nb + e] = (i < kb && j < kb && j >= i) ? T[i][j] : 0.0;
  }
}

// CT vectors per CTA, resident in shared memory for the whole product: vector c is
// X[i * xrs + c0 + c] (or e_{unit0 + c0 + c} when X is null) and leaves as out[i * ors + c0 + c]; X and
// out may be the same matrix (every CTA owns its columns). Blocks of reflectors, last block first, are
// staged in shared memory (zero where a reflector has no entry); a CTA with fewer than CT vectors pads
// with zero vectors, which stay zero.
template <int CT>
__global__ void __launch_bounds__(WY_THREADS, 1)
    wy_apply_kernel(const double* __restrict__ V, int64_t ldv, int off, int rel, const double* __restrict__ tau, int K,
                    int L, int nb, const double* __restrict__ Tg, const double* X, int64_t xrs, int64_t unit0, int nvec,
                    double* out, int64_t ors) {
  extern __shared__ double sm[];
  double* xs = sm;                       // CT x L: vector c at xs + c * L
  double* vs = sm + (size_t)CT * L;      // nb x L: reflector k0 + j at vs + j * L (rows >= k0 + off)
  __shared__ double Ts[WY_NB * WY_NB];
  __shared__ double Ws[WY_NB * CT], W2[WY_NB * CT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int c0 = blockIdx.x * CT;
  const int nc = min(CT, nvec - c0);
  for (int e = threadIdx.x; e < CT * L; e += blockDim.x) {
    const int i = e / CT, c = e - i * CT;
    double v = 0.0;
    if (c < nc) v = X ? X[(int64_t)i * xrs + c0 + c] : ((int64_t)i == unit0 + c0 + c ? 1.0 : 0.0);
    xs[(size_t)c * L + i] = v;
  }
  const int nblk = (K + nb - 1) / nb;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * nb, kb = min(nb, K - k0), i0 = k0 + off, span = L - i0;
    __syncthreads();  // the vectors are loaded / the previous block is applied
    if (span <= 0) continue;
    // eight loads in flight per thread before their stores (one at a time, each waited for the L2)
    const int tot = kb * span;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * WY_THREADS) {
      double val[8];
      int dst[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * WY_THREADS;
        val[u] = 0.0;
        dst[u] = -1;
        if (e < tot) {
          const int j = e / span, i = i0 + (e - j * span), k = k0 + j;
          dst[u] = j * L + i;
          if (i >= k + off && tau[k] != 0.0) val[u] = V[refl_index(ldv, off, rel, k, i)];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (dst[u] >= 0) vs[dst[u]] = val[u];
    }
    for (int e = threadIdx.x; e < nb * nb; e += WY_THREADS) Ts[e] = Tg[(int64_t)b * nb * nb + e];
    __syncthreads();
    // w = V^T x: one warp per reflector, every vector of the CTA in the same pass over v
    for (int j = warp; j < kb; j += nw) {
      double acc[CT];
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[c] = 0.0;
      const double* vj = vs + (size_t)j * L;
      for (int i = i0 + lane; i < L; i += 32) {
        const double v = vj[i];
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[c] = fma(v, xs[(size_t)c * L + i], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        const double sum = warp_sum(acc[c]);
        if (lane == 0) Ws[j * CT + c] = sum;
      }
    }
    __syncthreads();
    // w <- T w
    for (int e = threadIdx.x; e < kb * CT; e += blockDim.x) {
      const int a = e / CT, c = e - a * CT;
      double acc = 0.0;
      for (int l = a; l < kb; ++l) acc = fma(Ts[a * nb + l], Ws[l * CT + c], acc);
      W2[a * CT + c] = acc;
    }
    __syncthreads();
    // x -= V w on the rows the block touches
    for (int i = i0 + threadIdx.x; i < L; i += blockDim.x) {
      double acc[CT];
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[c] = 0.0;
      for (int j = 0; j < kb; ++j) {
        const double v = vs[(size_t)j * L + i];
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[c] = fma(v, W2[j * CT + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < CT; ++c) xs[(size_t)c * L + i] -= acc[c];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < CT * L; e += blockDim.x) {
    const int i = e / CT, c = e - i * CT;
    if (c < nc) out[(int64_t)i * ors + c0 + c] = xs[(size_t)c * L + i];
  }
}

template <int CT>
cudaError_t launch_apply_ct(const double* V, int64_t ldv, int off, int rel, const double* tau, int K, int L, int nb,
                            const double* Tg, const double* X, int64_t xrs, int64_t unit0, int nvec, double* out,
                            int64_t ors, cudaStream_t s) {
  const size_t sm = sizeof(double) * (size_t)L * (size_t)(CT + nb);
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(wy_apply_kernel<CT>));
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((nvec + CT - 1) / CT);
  wy_apply_kernel<CT><<<grid, WY_THREADS, sm, s>>>(V, ldv, off, rel, tau, K, L, nb, Tg, X, xrs, unit0, nvec, out, ors);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

size_t wy_workspace_bytes(int64_t K) { return sizeof(double) * (size_t)(WY_NB * K + WY_NB * WY_NB) + 256; }

cudaError_t launch_wy_apply(const double* V, int64_t ldv, int off, int rel, const double* tau, int64_t K, int64_t L,
                            const double* X, int64_t xrs, int64_t unit0, int64_t nvec, double* out, int64_t ors,
                            void* work, cudaStream_t s) {
  if (K < 1 || L < 1 || L > 4096 || K > L || nvec < 1 || off < 0 || off > 1 || rel < 0 || rel > 1)
    return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  nsm = std::max(nsm, 1);
  // rows of length L that fit in about 200 KB of shared memory: the vectors plus one block of reflectors
  const int64_t rows_fit = (200 * 1024) / (8 * L);
  // vectors per CTA: few enough that the CTAs cover every SM, at most 8, and leaving room for reflectors
  static const int kCT[] = {1, 2, 3, 4, 6, 8};
  const int64_t spread = (nvec + nsm - 1) / nsm;
  int ct = 1;
  for (int c : kCT)
    if (c + 1 <= rows_fit) {
      ct = c;
      if (c >= spread) break;
    }
  const int nb = (int)std::min<int64_t>({(int64_t)WY_NB, rows_fit - ct, K});
  if (nb < 1) return cudaErrorInvalidValue;
  double* Tg = static_cast<double*>(work);
  const int nblk = (int)((K + nb - 1) / nb);
  wy_tfactor_kernel<<<nblk, WY_THREADS, 0, s>>>(V, ldv, off, rel, tau, (int)K, (int)L, nb, Tg);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int Ki = (int)K, Li = (int)L, nv = (int)nvec;
  switch (ct) {
    case 1: return launch_apply_ct<1>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
    case 2: return launch_apply_ct<2>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
    case 3: return launch_apply_ct<3>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
    case 4: return launch_apply_ct<4>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
    case 6: return launch_apply_ct<6>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
    default: return launch_apply_ct<8>(V, ldv, off, rel, tau, Ki, Li, nb, Tg, X, xrs, unit0, nv, out, ors, s);
  }
}

}  // namespace bht

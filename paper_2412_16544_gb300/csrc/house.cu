// house.cu — orthonormal complement of orthonormal columns by Householder QR.
//
// For Z (c x k) with orthonormal columns, the QR factorisation
// Z = H_0 H_1 ... H_{k-1} [R; 0] gives an orthogonal c x c matrix whose first
// k columns span Z and whose last c - k columns are an orthonormal basis of
// the complement. HT-RISE keeps that complement for each node (the residual
// of a later batch lives in it); after an expansion by k directions Z inside
// the old complement Q (a x c), the new complement is
// Q H_0 ... H_{k-1} restricted to its last c - k columns.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "sync.cuh"

namespace bht {

namespace {

constexpr int HQ_THREADS = 256;

// Householder QR of Z (c x k, row-major, ld k) with the rows resident in shared memory: row i
// belongs to CTA i % gridDim.x (slot i / gridDim.x). Step j needs the squared norm of column j
// below the diagonal and v_j^T Z(:, q) for the later columns q; with v_j = (x - beta e_j) / (alpha
// - beta) (x = column j from row j on, alpha = Z(j, j)) the latter is Z(j, q) + scale h_q with
// h_q = sum_{i > j} Z(i, j) Z(i, q), and the former is h_j. So one reduction per column, of h over
// q >= j, suffices: every CTA adds its rows' products into h (FP64 atomics) right after it has
// applied the previous reflector, the owner of row j publishes that row, and after one grid barrier
// every CTA forms the same reflector and the same v_j^T Z. The sums rotate through three buffers
// (read at step j, accumulated for step j + 1, cleared for step j + 2) and the published row through
// two. V[j * c + i] receives v_j[i] (zero above the diagonal).
// Work buffers: hsum[3][k] (zero on entry), prow[2][k].
__global__ void __launch_bounds__(HQ_THREADS) house_qr_kernel(const double* __restrict__ Z, int c, int k, int rpb,
                                                              double* __restrict__ V, double* __restrict__ tau,
                                                              double* __restrict__ hsum, double* __restrict__ prow,
                                                              Barrier* bar, int* status) {
  extern __shared__ double sm[];
  double* rows = sm;                       // rpb x k
  double* dv = rows + (size_t)rpb * k;     // k: v_j^T Z(:, q)
  double* zq = dv + k;                     // k: the published pivot row
  double* vloc = zq + k;                   // rpb: v_j on the own rows
  __shared__ double scal[2];               // tau_j and 1 / (alpha - beta) of the step
  const int nb = gridDim.x, b = blockIdx.x;
  unsigned int epoch = 0;  // barriers passed (grid_barrier_count)
  for (int l = 0; l < rpb; ++l) {
    const int i = b + l * nb;
    for (int q = threadIdx.x; q < k; q += blockDim.x) rows[(size_t)l * k + q] = (i < c) ? Z[(size_t)i * k + q] : 0.0;
  }
  __syncthreads();
  // sums for column 0 and the published row 0
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double h = 0.0;
    for (int l = 0; l < rpb; ++l) {
      const int i = b + l * nb;
      if (i > 0 && i < c) h = fma(rows[(size_t)l * k], rows[(size_t)l * k + q], h);
    }
    if (h != 0.0) atomicAdd(&hsum[q], h);
    if (b == 0) prow[q] = rows[q];  // row 0 lives in slot 0 of CTA 0
  }
  if (!grid_barrier_count(bar, epoch, status)) return;
  for (int j = 0; j < k; ++j) {
    const double* h = hsum + (size_t)(j % 3) * k;
    const double* zr = prow + (size_t)(j & 1) * k;
    // this step's sums and pivot row for the later columns, fetched while thread 0 forms the reflector
    for (int q = j + 1 + threadIdx.x; q < k; q += blockDim.x) {
      dv[q] = h[q];
      zq[q] = zr[q];
    }
    // the reflector, identical in every CTA (same sums); its scalar FP64 chain runs on thread 0 only
    // (run by every warp it would hold each SM sub-partition's FP64 pipe 64 cycles per instruction)
    if (threadIdx.x == 0) {
      const double alpha = zr[j], xn2 = h[j];
      double t0 = 0.0, s0 = 0.0;
      if (xn2 > 0.0) {
        const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        // tj = (beta - alpha) / beta and scale = 1 / (alpha - beta) from one reciprocal of their product
        const double am = alpha - beta, inv = 1.0 / (beta * am);
        t0 = -am * am * inv;
        s0 = beta * inv;
      }
      scal[0] = t0;
      scal[1] = s0;
    }
    __syncthreads();
    const double tj = scal[0], scale = scal[1];
    for (int q = j + 1 + threadIdx.x; q < k; q += blockDim.x) dv[q] = fma(scale, dv[q], zq[q]);  // own entries
    for (int l = threadIdx.x; l < rpb; l += blockDim.x) {
      const int i = b + l * nb;
      double v = 0.0;
      if (i == j) v = 1.0;
      else if (i > j && i < c) v = (tj != 0.0) ? rows[(size_t)l * k + j] * scale : 0.0;
      vloc[l] = v;
      if (i < c) V[(size_t)j * c + i] = v;
    }
    if (b == 0) {
      if (threadIdx.x == 0) tau[j] = tj;
      double* clr = hsum + (size_t)((j + 2) % 3) * k;  // the buffer of step j + 2
      for (int q = threadIdx.x; q < k; q += blockDim.x) clr[q] = 0.0;
    }
    __syncthreads();
    // Z(:, q) -= (tau v_i) (v^T Z(:, q)) on the own rows, q > j: one FMA per entry
    if (tj != 0.0) {
      for (int l = 0; l < rpb; ++l) {
        const double tv = tj * vloc[l];
        if (tv == 0.0) continue;
        double* row = rows + (size_t)l * k;
        for (int q = j + 1 + threadIdx.x; q < k; q += blockDim.x) row[q] = fma(-tv, dv[q], row[q]);
      }
    }
    __syncthreads();
    // sums for column j + 1 from the updated rows, and row j + 1 published by its owner
    if (j + 1 < k) {
      double* hn = hsum + (size_t)((j + 1) % 3) * k;
      double* pr = prow + (size_t)((j + 1) & 1) * k;
      const int jn = j + 1;
      const bool owner = (jn % nb) == b;
      const int lo = jn / nb;
      for (int q = jn + threadIdx.x; q < k; q += blockDim.x) {
        double hq = 0.0;
        for (int l = 0; l < rpb; ++l) {
          const int i = b + l * nb;
          if (i > jn && i < c) hq = fma(rows[(size_t)l * k + jn], rows[(size_t)l * k + q], hq);
        }
        if (hq != 0.0) atomicAdd(&hn[q], hq);
        if (owner) pr[q] = rows[(size_t)lo * k + q];
      }
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
  }
}

// out[m][0 .. c-k) = (Q[m] H_0 H_1 ... H_{k-1})[k .. c) for every row m of Q (a x c): one warp per
// row, a CTA's rows staged in shared memory together with blocks of nbr reflectors, each block loaded
// once per CTA (coalesced) for all its warps. With many rows the warps keep the FP64 pipe busy; the
// complement of Z itself (Q the identity) goes through the blocked form in wy.cu instead.
__global__ void __launch_bounds__(HQ_THREADS) apply_reflectors_kernel(const double* __restrict__ Q, int64_t a, int c,
                                                                      int k, int nbr, const double* __restrict__ V,
                                                                      const double* __restrict__ tau,
                                                                      double* __restrict__ out) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double* q = sm + (size_t)w * c;
  double* vb = sm + (size_t)nwarp * c;  // nbr reflectors, row (j - j0) holds v_j
  const int64_t nbatch = (a + nwarp - 1) / nwarp;
  for (int64_t bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const int64_t m = bt * nwarp + w;
    const bool act = m < a;
    __syncthreads();  // the previous batch's rows are written out
    if (act)
      for (int i = lane; i < c; i += 32) q[i] = Q[m * c + i];
    for (int j0 = 0; j0 < k; j0 += nbr) {
      const int j1 = min(k, j0 + nbr);
      __syncthreads();  // the previous reflector block is consumed
      for (int jj = j0; jj < j1; ++jj) {
        const double* src = V + (size_t)jj * c;
        double* dst = vb + (size_t)(jj - j0) * c;
        for (int i = jj + threadIdx.x; i < c; i += blockDim.x) dst[i] = src[i];
      }
      __syncthreads();
      if (!act) continue;
      for (int j = j0; j < j1; ++j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        const double* v = vb + (size_t)(j - j0) * c;
        double d = 0.0;
        for (int i = j + lane; i < c; i += 32) d = fma(q[i], v[i], d);
        d = warp_sum(d) * tj;
        for (int i = j + lane; i < c; i += 32) q[i] -= d * v[i];
        __syncwarp();
      }
    }
    if (act)
      for (int i = k + lane; i < c; i += 32) out[m * (c - k) + (i - k)] = q[i];
  }
}

}  // namespace

// V [k][c], tau [k], hsum [3][k], prow [2][k], the barrier word, then the block factors of the
// blocked application (identity case), 256-byte aligned.
static size_t house_barrier_offset(int64_t c, int64_t k) { return sizeof(double) * ((size_t)k * c + 6 * (size_t)k); }
static size_t house_factors_offset(int64_t c, int64_t k) {
  return (house_barrier_offset(c, k) + sizeof(Barrier) + 255) & ~(size_t)255;
}

size_t house_workspace_bytes(int64_t c, int64_t k, int nsm) {
  (void)nsm;
  return house_factors_offset(c, k) + wy_workspace_bytes(k) + 256;
}

cudaError_t launch_house_complement(const double* Q, int64_t a, int64_t c, const double* Z, int64_t k, double* out,
                                    void* work, int* status, cudaStream_t s) {
  if (k <= 0 || c <= k || a <= 0 || (!Q && a != c)) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // about 8 rows per CTA, at most one CTA per SM, the rows in shared memory
  int rpb = (int)std::max<int64_t>(8, (c + nsm - 1) / nsm);
  const int nb = (int)((c + rpb - 1) / rpb);
  const size_t smq = sizeof(double) * ((size_t)rpb * k + 2 * (size_t)k + rpb);
  if (smq > 200 * 1024) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(work);
  double* V = reinterpret_cast<double*>(p);
  double* tau = V + (size_t)k * c;
  double* hsum = tau + k;
  double* prow = hsum + 3 * (size_t)k;
  Barrier* bar = reinterpret_cast<Barrier*>(p + house_barrier_offset(c, k));  // = prow + 2k
  cudaError_t e = cudaMemsetAsync(hsum, 0, sizeof(double) * 5 * (size_t)k + sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  if (smq > 0) {  // dynamic + static must fit the cap
    e = allow_max_smem(reinterpret_cast<const void*>(house_qr_kernel));
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope prof(K_HOUSE, s, 4.0 * (double)c * (double)k * (double)k, 8.0 * (double)c * (double)k * 2.0);
    int ci = (int)c, ki = (int)k;
    void* args[] = {&Z, &ci, &ki, &rpb, &V, &tau, &hsum, &prow, &bar, &status};
    if (nb == 1) {
      house_qr_kernel<<<1, HQ_THREADS, smq, s>>>(Z, ci, ki, rpb, V, tau, hsum, prow, bar, status);
      e = cudaGetLastError();
    } else {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, house_qr_kernel, HQ_THREADS, smq);
      if (e != cudaSuccess) return e;
      if ((int64_t)per_sm * nsm < nb) return cudaErrorInvalidConfiguration;
      e = cudaLaunchCooperativeKernel((void*)house_qr_kernel, dim3(nb), dim3(HQ_THREADS), args, smq, s);
    }
    note_launch();
    if (e != cudaSuccess) return e;
  }
  if (!Q) {
    // the complement itself: H_0 ... H_{k-1} applied to e_k .. e_{c-1} in blocks of reflectors (wy.cu),
    // c - k vectors instead of the c rows of the identity
    ProfScope prof(K_HOUSE, s, 2.0 * (double)(c - k) * (2.0 * (double)c * (double)k - (double)k * (double)k),
                   8.0 * (double)c * ((double)k + (double)(c - k)));
    return launch_wy_apply(V, c, 0, 0, tau, k, c, nullptr, 0, k, c - k, out, c - k, p + house_factors_offset(c, k), s);
  }
  // rows of one CTA plus a block of reflectors, about 200 KB at most
  const int nwarp = HQ_THREADS / 32;
  const int nbr = (int)std::max<int64_t>(1, std::min<int64_t>(32, (200 * 1024) / (8 * c) - nwarp));
  const size_t sma = sizeof(double) * (size_t)c * (nwarp + nbr);
  if (sma > 200 * 1024) return cudaErrorInvalidValue;
  if (sma > 0) {  // dynamic + static must fit the cap
    e = allow_max_smem(reinterpret_cast<const void*>(apply_reflectors_kernel));
    if (e != cudaSuccess) return e;
  }
  ProfScope prof(K_HOUSE, s, 4.0 * (double)a * (double)c * (double)k, 8.0 * (double)a * (double)c * 2.0);
  const int blocks = (int)std::min<int64_t>((a + nwarp - 1) / nwarp, (int64_t)nsm * 2);
  apply_reflectors_kernel<<<blocks, HQ_THREADS, sma, s>>>(Q, a, (int)c, (int)k, nbr, V, tau, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

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

// Householder QR of Z (c x k, row-major, ld k) with the rows resident in shared
// memory: row i belongs to CTA i % gridDim.x (slot i / gridDim.x). Column j:
// the CTAs publish partial squared norms below the diagonal and the diagonal
// entry, pass a grid barrier, every CTA forms the same reflector
// v_j (v_j[j] = 1) and tau_j, adds its partial products v_j^T Z(:, l) for the
// later columns into dsum (FP64 atomics), passes a second barrier and updates
// its rows. V[j * c + i] receives v_j[i] (zero above the diagonal).
// Work buffers: part[2][gridDim.x], diag[2], dsum[2][k] (zero on entry).
__global__ void __launch_bounds__(HQ_THREADS) house_qr_kernel(const double* __restrict__ Z, int c, int k, int rpb,
                                                              double* __restrict__ V, double* __restrict__ tau,
                                                              double* __restrict__ part, double* __restrict__ diag,
                                                              double* __restrict__ dsum, Barrier* bar, int* status) {
  extern __shared__ double sm[];
  double* rows = sm;                     // rpb x k
  double* vloc = rows + (size_t)rpb * k;  // rpb: v_j on the own rows
  __shared__ double red[33];
  const int nb = gridDim.x, b = blockIdx.x;
  unsigned int epoch = 0;  // barriers passed (grid_barrier_count)
  for (int l = 0; l < rpb; ++l) {
    const int i = b + l * nb;
    for (int q = threadIdx.x; q < k; q += blockDim.x) rows[(size_t)l * k + q] = (i < c) ? Z[(size_t)i * k + q] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const int par = j & 1;
    // A: partial ||Z(j+1:, j)||^2 and the diagonal entry
    double s = 0.0;
    for (int l = threadIdx.x; l < rpb; l += blockDim.x) {
      const int i = b + l * nb;
      const double z = rows[(size_t)l * k + j];
      if (i > j && i < c) s = fma(z, z, s);
      if (i == j) diag[par] = z;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[par * nb + b] = s;
    if (!grid_barrier_count(bar, epoch, status)) return;
    // B: the reflector, identical in every CTA (same partials, same order)
    double t = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) t += part[par * nb + q];
    const double xn2 = block_sum(t, red);
    const double alpha = diag[par];
    double tj = 0.0, scale = 0.0;
    if (xn2 > 0.0) {
      const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
      tj = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
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
      for (int q = threadIdx.x; q < k; q += blockDim.x) dsum[(par ^ 1) * k + q] = 0.0;  // next column's sums
    }
    __syncthreads();
    if (tj != 0.0) {
      for (int q = j + 1 + threadIdx.x; q < k; q += blockDim.x) {
        double d = 0.0;
        for (int l = 0; l < rpb; ++l) d = fma(vloc[l], rows[(size_t)l * k + q], d);
        if (d != 0.0) atomicAdd(&dsum[par * k + q], d);
      }
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
    // C: Z(:, q) -= tau v (v^T Z(:, q)) on the own rows
    if (tj != 0.0) {
      for (int e = threadIdx.x; e < rpb * (k - j - 1); e += blockDim.x) {
        const int l = e / (k - j - 1), q = j + 1 + e % (k - j - 1);
        const double v = vloc[l];
        if (v != 0.0) rows[(size_t)l * k + q] -= tj * v * dsum[par * k + q];
      }
    }
    __syncthreads();
  }
}

// out[m][0 .. c-k) = (Q[m] H_0 H_1 ... H_{k-1})[k .. c) for every row m of Q (a x c):
// one warp per row, the row staged in shared memory.
__global__ void __launch_bounds__(HQ_THREADS) apply_reflectors_kernel(const double* __restrict__ Q, int64_t a, int c,
                                                                      int k, const double* __restrict__ V,
                                                                      const double* __restrict__ tau,
                                                                      double* __restrict__ out) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* q = sm + (size_t)w * c;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; m < a; m += nw) {
    for (int i = lane; i < c; i += 32) q[i] = Q[m * c + i];
    __syncwarp();
    for (int j = 0; j < k; ++j) {
      const double tj = tau[j];
      if (tj == 0.0) continue;
      const double* v = V + (size_t)j * c;
      double d = 0.0;
      for (int i = j + lane; i < c; i += 32) d = fma(q[i], v[i], d);
      d = warp_sum(d) * tj;
      for (int i = j + lane; i < c; i += 32) q[i] -= d * v[i];
      __syncwarp();
    }
    for (int i = k + lane; i < c; i += 32) out[m * (c - k) + (i - k)] = q[i];
    __syncwarp();
  }
}

}  // namespace

size_t house_workspace_bytes(int64_t c, int64_t k, int nsm) {
  return sizeof(double) * ((size_t)k * c + k + 2 * (size_t)nsm + 2 + 2 * (size_t)k) + 2 * 256 + sizeof(Barrier);
}

cudaError_t launch_house_complement(const double* Q, int64_t a, int64_t c, const double* Z, int64_t k, double* out,
                                    void* work, int* status, cudaStream_t s) {
  if (k <= 0 || c <= k || a <= 0) return cudaErrorInvalidValue;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // about 8 rows per CTA, at most one CTA per SM, the rows in shared memory
  int rpb = (int)std::max<int64_t>(8, (c + nsm - 1) / nsm);
  const int nb = (int)((c + rpb - 1) / rpb);
  const size_t smq = sizeof(double) * ((size_t)rpb * k + rpb);
  if (smq > 200 * 1024) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(work);
  double* V = reinterpret_cast<double*>(p);
  double* tau = V + (size_t)k * c;
  double* part = tau + k;
  double* diag = part + 2 * (size_t)nsm;
  double* dsum = diag + 2;
  Barrier* bar = reinterpret_cast<Barrier*>(dsum + 2 * (size_t)k);
  cudaError_t e = cudaMemsetAsync(dsum, 0, sizeof(double) * 2 * (size_t)k + sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  if (smq > 48 * 1024) {
    e = cudaFuncSetAttribute(house_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq);
    if (e != cudaSuccess) return e;
  }
  {
    ProfScope prof(K_HOUSE, s, 4.0 * (double)c * (double)k * (double)k, 8.0 * (double)c * (double)k * 2.0);
    int ci = (int)c, ki = (int)k;
    void* args[] = {&Z, &ci, &ki, &rpb, &V, &tau, &part, &diag, &dsum, &bar, &status};
    if (nb == 1) {
      house_qr_kernel<<<1, HQ_THREADS, smq, s>>>(Z, ci, ki, rpb, V, tau, part, diag, dsum, bar, status);
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
  const size_t sma = sizeof(double) * (size_t)c * (HQ_THREADS / 32);
  if (sma > 200 * 1024) return cudaErrorInvalidValue;
  if (sma > 48 * 1024) {
    e = cudaFuncSetAttribute(apply_reflectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma);
    if (e != cudaSuccess) return e;
  }
  ProfScope prof(K_HOUSE, s, 4.0 * (double)a * (double)c * (double)k, 8.0 * (double)a * (double)c * 2.0);
  const int blocks = (int)std::min<int64_t>((a + 7) / 8, (int64_t)nsm * 4);
  apply_reflectors_kernel<<<blocks, HQ_THREADS, sma, s>>>(Q, a, (int)c, (int)k, V, tau, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

// eig.cu — FP64 symmetric eigensolver for the node truncations.
//
// The error-truncated SVD of a node unfolding (eq. ht_leaf_svd, eq.
// svd_on_residual) keeps the left singular vectors: they are the eigenvectors
// of the unfolding's Gram matrix, with eigenvalues sigma_i^2. The truncation
// rank only needs all eigenvalues, and the node only needs the eigenvectors it
// keeps, so the solver runs in two stages:
//   stage 1  Householder tridiagonalisation Q^T G Q = T, then every eigenvalue
//            of T by Sturm-sequence multisection (16 or 32 points per round);
//   stage 2  (after the caller picked r) the eigenvectors of T for the r
//            largest eigenvalues by twisted factorisation (one thread per
//            eigenvalue; one CTA per cluster of nearly equal eigenvalues
//            orthogonalises its members), then the back-transformation U = Q Z.
// GB300 has few FP64 units (about 2 FMA per clock per SM), so every stage is
// spread over the whole GPU: the tridiagonalisation keeps the matrix rows in
// the shared memory of one cooperative grid (one CTA for n <= 64) with one
// bounded grid barrier per column; matrices too large for that fall back to a
// global-memory form with two barriers per column.
#include <algorithm>
#include <cfloat>
#include <cstdlib>
#include <atomic>
#include <mutex>
#include <vector>
#include <cmath>

#include "bht.h"
#include "internal.cuh"
#include "sync.cuh"

namespace bht {

namespace {

constexpr int EIG_THREADS = 256;
constexpr int SMALL_N = 16;
constexpr int ONE_CTA_N = 64;  // the row-resident tridiagonalisation runs in one CTA up to this size: its
                               // per-column FP64 work (2 n^2 FMAs) stays below a grid barrier's latency

// ---------------------------------------------------------------------------
// Householder tridiagonalisation of the symmetric matrix A (n x n, both
// triangles kept up to date). Step k maps column k below the diagonal onto
// beta e_1 with H_k = I - tau_k v_k v_k^T, v_k[0] = 1 (stored in Vh row k):
//   p = tau A22 v,  w = p - (tau/2)(p.v) v,  A22 -= v w^T + w v^T.
// Every CTA recomputes v (and w) from the same data, so only p is exchanged.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EIG_THREADS) tridiag_kernel(double* __restrict__ A, int n,
                                                              double* __restrict__ Vh, double* __restrict__ d,
                                                              double* __restrict__ e, double* __restrict__ tau,
                                                              double* __restrict__ pbuf, Barrier* bar,
                                                              int* status) {
  extern __shared__ double sm[];
  unsigned int epoch = 0;  // barriers passed (grid_barrier_count)
  double* v = sm;       // n
  double* w = sm + n;   // n
  __shared__ double red[33];
  __shared__ double sc[3];
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;

  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const double* rowk = A + (int64_t)k * n + k + 1;  // = column k below the diagonal
    double s = 0.0;
    for (int j = 1 + threadIdx.x; j < m; j += blockDim.x) s = fma(rowk[j], rowk[j], s);
    const double xn2 = block_sum(s, red);
    if (threadIdx.x == 0) {
      const double alpha = rowk[0];
      double t = 0.0, beta = alpha, scale = 0.0;
      if (xn2 > 0.0) {
        beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        t = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
      sc[0] = t;
      sc[1] = beta;
      sc[2] = scale;
    }
    __syncthreads();
    const double tk = sc[0], scale = sc[2];
    for (int j = threadIdx.x; j < m; j += blockDim.x) v[j] = (j == 0) ? 1.0 : (tk != 0.0 ? rowk[j] * scale : 0.0);
    if (blockIdx.x == 0) {
      for (int j = threadIdx.x; j < m; j += blockDim.x) Vh[(int64_t)k * n + j] = v[j];
      if (threadIdx.x == 0) {
        d[k] = A[(int64_t)k * n + k];
        e[k] = sc[1];
        tau[k] = tk;
      }
    }
    __syncthreads();
    if (tk == 0.0) {  // column already reduced: no reflection, nothing to update
      if (!grid_barrier_count(bar, epoch, status)) return;
      continue;
    }
    // p = tau A22 v, one warp per row
    const int64_t base = (int64_t)(k + 1) * n + (k + 1);
    for (int i = gwarp; i < m; i += nwarps) {
      const double* row = A + base + (int64_t)i * n;
      double dot = 0.0;
      for (int j = lane; j < m; j += 32) dot = fma(row[j], v[j], dot);
      dot = warp_sum(dot);
      if (lane == 0) pbuf[i] = tk * dot;
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
    // w = p - (tau/2)(p.v) v
    double pv = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double pj = pbuf[j];
      w[j] = pj;
      pv = fma(pj, v[j], pv);
    }
    const double K = 0.5 * tk * block_sum(pv, red);
    for (int j = threadIdx.x; j < m; j += blockDim.x) w[j] -= K * v[j];
    __syncthreads();
    // A22 -= v w^T + w v^T, one warp per row
    for (int i = gwarp; i < m; i += nwarps) {
      double* row = A + base + (int64_t)i * n;
      const double vi = v[i], wi = w[i];
      for (int j = lane; j < m; j += 32) row[j] -= vi * w[j] + wi * v[j];
    }
    if (!grid_barrier_count(bar, epoch, status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = A[(int64_t)(n - 2) * n + (n - 2)];
      e[n - 2] = A[(int64_t)(n - 1) * n + (n - 2)];
      tau[n - 2] = 0.0;
    }
    d[n - 1] = A[(int64_t)(n - 1) * n + (n - 1)];
    e[n - 1] = 0.0;
    tau[n - 1] = 0.0;
  }
}

// Householder reflector of x[0..m) (m >= 2), computed by every thread of the
// block: v[0] = 1, v[j] = x[j] / (x[0] - beta), tau = (beta - x[0]) / beta,
// H x = beta e_1. Returns tau; *beta_out receives beta. x and v in shared memory.
__device__ double householder(const double* x, int m, double* v, double* red, double* beta_out) {
  double s = 0.0;
  for (int j = 1 + threadIdx.x; j < m; j += blockDim.x) s = fma(x[j], x[j], s);
  const double xn2 = block_sum(s, red);
  const double alpha = x[0];
  double t = 0.0, beta = alpha, scale = 0.0;
  if (xn2 > 0.0) {
    beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
    // t = (beta - alpha) / beta and scale = 1 / (alpha - beta) from one reciprocal of their product
    const double am = alpha - beta, inv = 1.0 / (beta * am);
    t = -am * am * inv;
    scale = beta * inv;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) v[j] = (j == 0) ? 1.0 : (t != 0.0 ? x[j] * scale : 0.0);
  *beta_out = beta;
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// Householder tridiagonalisation with the matrix resident in shared memory.
// Row gi belongs to CTA gi % gridDim.x (slot gi / gridDim.x) for the whole
// reduction, so the rank-2 updates and matrix-vector products never leave the
// SM. One grid barrier (a growing counter) per column: after it every CTA holds p_t = tau A22 v_t
// and row t+1 as it was before update t (published by its owner), and itself
// forms w_t, the updated column t+1 and the next reflector v_{t+1}; then one
// pass over its rows applies update t and accumulates p_{t+1} at once.
// p and the published row alternate between two buffers by column parity.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EIG_THREADS) tridiag_rows_kernel(const double* __restrict__ A, int n, int rpb,
                                                                   double* __restrict__ Vh, double* __restrict__ d,
                                                                   double* __restrict__ e, double* __restrict__ tau,
                                                                   double* __restrict__ pbuf, double* __restrict__ pub,
                                                                   Barrier* bar, int* status) {
  extern __shared__ double sm[];
  double* rows = sm;                         // rpb x n
  double* vb[2] = {rows + (size_t)rpb * n, rows + (size_t)(rpb + 1) * n};
  double* w = rows + (size_t)(rpb + 2) * n;  // n
  double* x = rows + (size_t)(rpb + 3) * n;  // n
  __shared__ double red[33];
  __shared__ double scal[4];  // K_t, tau_{t+1}, 1 / (alpha - beta) of the step
  const int nb = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int epoch = 0;  // barriers passed (grid_barrier_count)
  const unsigned int bflags = (threadIdx.x == 0) ? bar->flags : 0u;  // test hooks of the barrier (zero normally)
  for (int l = 0; l < rpb; ++l) {
    const int gi = b + l * nb;
    if (gi >= n) break;
    for (int j = threadIdx.x; j < n; j += blockDim.x) rows[(size_t)l * n + j] = A[(size_t)gi * n + j];
  }
  // column 0: reflector from row 0, p_0 from the own rows
  for (int j = threadIdx.x; j < n - 1; j += blockDim.x) x[j] = A[j + 1];
  __syncthreads();
  double beta = 0.0;
  double tc = householder(x, n - 1, vb[0], red, &beta);
  if (b == 0) {
    for (int j = threadIdx.x; j < n - 1; j += blockDim.x) Vh[j] = vb[0][j];
    if (threadIdx.x == 0) {
      d[0] = A[0];
      e[0] = beta;
      tau[0] = tc;
    }
  }
  for (int l = warp; l < rpb; l += nw) {
    const int gi = b + l * nb;
    if (gi < 1 || gi >= n) continue;
    const double* r = rows + (size_t)l * n;
    double dot = 0.0;
    for (int c = 1 + lane; c < n; c += 32) dot = fma(r[c], vb[0][c - 1], dot);
    dot = warp_sum(dot);
    if (lane == 0) pbuf[gi - 1] = tc * dot;
    if (gi == 1)
      for (int c = 1 + lane; c < n; c += 32) pub[n + c] = r[c];
  }
  if (!grid_barrier_count(bar, epoch, status, bflags)) return;

  for (int t = 0; t + 2 < n; ++t) {
    const int m = n - t - 1;  // length of v_t; index q <-> column t + 1 + q
    const double* v = vb[t & 1];
    double* vn = vb[(t + 1) & 1];
    const double* p = pbuf + (size_t)(t & 1) * n;
    const double* R = pub + (size_t)((t + 1) & 1) * n;  // row t + 1 before update t
    // w_t = p - (tau/2)(p.v) v; row t + 1 is fetched in the same pass (both come from L2 after the
    // barrier, so their latencies overlap)
    double pv = 0.0;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
      const double pq = p[q];
      w[q] = pq;
      if (q >= 1) x[q - 1] = R[t + 1 + q];
      pv = fma(pq, v[q], pv);
    }
    // The second levels of the two reductions and every scalar of the step run on thread 0, which
    // publishes them in shared memory: a scalar FP64 chain executed by every warp would hold each SM
    // sub-partition's FP64 pipe for 64 cycles per instruction and per warp, and the rows' updates need it.
    pv = warp_sum(pv);
    if (lane == 0) red[warp] = pv;
    __syncthreads();
    if (warp == 0) {  // the warps' partial sums in log2(nw) shuffle steps, the scalar on lane 0
      const double sum = warp_sum_first(lane < nw ? red[lane] : 0.0, nw);
      if (lane == 0) scal[0] = 0.5 * tc * sum;
    }
    __syncthreads();
    const double Kc = scal[0];
    for (int q = threadIdx.x; q < m; q += blockDim.x) w[q] -= Kc * v[q];
    __syncthreads();
    // column t + 1 after update t: x[c - t - 2] for columns c >= t + 2 (each thread the entries it
    // fetched above), with the squared norm below its first entry
    const int m1 = m - 1;
    double xs = 0.0;
    for (int q = 1 + threadIdx.x; q < m; q += blockDim.x) {
      const double xq = x[q - 1] - (w[q] + w[0] * v[q]);
      x[q - 1] = xq;
      if (q >= 2) xs = fma(xq, xq, xs);
    }
    xs = warp_sum(xs);
    if (lane == 0) red[warp] = xs;
    __syncthreads();
    const double xn2 = (warp == 0) ? warp_sum_first(lane < nw ? red[lane] : 0.0, nw) : 0.0;
    if (threadIdx.x == 0) {
      // the reflector of column t + 1 (v[0] = 1), as in householder()
      const double alpha = x[0];
      double tt = 0.0, bt = alpha, sc = 0.0;
      if (m1 >= 2 && xn2 > 0.0) {
        bt = -copysign(sqrt(alpha * alpha + xn2), alpha);
        const double am = alpha - bt, inv = 1.0 / (bt * am);
        tt = -am * am * inv;
        sc = bt * inv;
      }
      scal[1] = tt;
      scal[2] = sc;
      if (b == 0) {
        d[t + 1] = R[t + 1] - 2.0 * w[0];
        e[t + 1] = bt;
        tau[t + 1] = tt;
      }
    }
    __syncthreads();
    const double tn = scal[1], vscale = scal[2];
    if (m1 >= 2) {
      for (int j = threadIdx.x; j < m1; j += blockDim.x) {
        const double vj = (j == 0) ? 1.0 : (tn != 0.0 ? x[j] * vscale : 0.0);
        vn[j] = vj;
        if (b == 0) Vh[(size_t)(t + 1) * n + j] = vj;
      }
    } else if (threadIdx.x == 0) {
      vn[0] = 1.0;
    }
    __syncthreads();
    // update t on the own rows gi >= t + 2, with p_{t+1} from the updated entries
    double* pn = pbuf + (size_t)((t + 1) & 1) * n;
    double* Rn = pub + (size_t)(t & 1) * n;  // row t + 2 after update t
    for (int l = warp; l < rpb; l += nw) {
      const int gi = b + l * nb;
      if (gi < t + 2 || gi >= n) continue;
      double* r = rows + (size_t)l * n;
      const int ig = gi - t - 1;
      const double vi = v[ig], wi = w[ig];
      const bool publish = (gi == t + 2);
      double dot = 0.0;
      for (int q = 1 + lane; q < m; q += 32) {
        const int c = t + 1 + q;
        const double a = fma(-vi, w[q], fma(-wi, v[q], r[c]));  // three FP64 operations per entry with the dot
        r[c] = a;
        dot = fma(a, vn[q - 1], dot);
        if (publish) Rn[c] = a;
      }
      if (m1 >= 2) {
        dot = warp_sum(dot);
        if (lane == 0) pn[gi - t - 2] = tn * dot;
      }
      if (gi == n - 1 && m1 < 2 && lane == 0) d[n - 1] = r[n - 1];
    }
    tc = tn;
    if (!grid_barrier_count(bar, epoch, status, bflags)) return;
  }
  if (b == 0 && threadIdx.x == 0) {
    e[n - 1] = 0.0;
    tau[n - 2] = 0.0;
    tau[n - 1] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Sturm-sequence multisection: every eigenvalue of the tridiagonal (d, e).
// ---------------------------------------------------------------------------
// The number of eigenvalues of T below x is the number of negative ratios
// q_i = p_i / p_{i-1} of the leading principal minors p_i of T - x I,
// p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}. The minors are carried instead
// of the ratios, so a step costs three FP64 operations (no division): FP64
// issues at 1/64 of the FP32 rate on this part and dominates the sweep. The
// sign test and the range test read the high word of p as an integer (sign
// bit and exponent field), off the FP64 pipe. T arrives scaled by a power of
// two so that |d_i|, |x| <= 2 and e_i^2 <= 4: one step grows |p| at most
// 8-fold, and whenever |p_i| leaves [2^-500, 2^500] both carried minors are
// rescaled by 2^-+500 (exact). An exactly zero minor becomes -2^-200 p_{i-1}:
// a zero pivot counts as negative.
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x) {
  double a0 = 1.0, a1 = d[0] - x;
  if (a1 == 0.0) a1 = -0x1p-200;
  int cnt = a1 < 0.0;
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    double t = fma(d[i] - x, a1, -e2[i - 1] * a0);
    const unsigned ex = ((unsigned)__double2hiint(t) >> 20) & 0x7FFu;
    if (ex - (1023u - 500u) > 1000u) {  // exponent outside [-500, 500], zero or subnormal
      if (t == 0.0) t = -0x1p-200 * a1;
      const double f = fabs(t) > 1.0 ? 0x1p-500 : 0x1p+500;
      if (fabs(t) > 0x1p+500 || fabs(t) < 0x1p-500) {
        t *= f;
        a1 *= f;
      }
    }
    cnt += (__double2hiint(t) ^ __double2hiint(a1)) < 0;
    a0 = a1;
    a1 = t;
  }
  return cnt;
}

// The same count in FP32 (the FP32 pipe issues 64 times faster than the FP64 one on this part), with
// the carried minors kept within [2^-40, 2^40] and an exactly zero minor replaced by -2^-60 p_{i-1}.
// With unit roundoff u = 2^-24, each step's three roundings and the rounding of d_i, e_i^2 and x to
// FP32 make the count exact for a tridiagonal matrix T' with |d'_i - d_i| <= 2u (|d_i| + |x|) and
// |e'_i - e_i| <= 1.5u |e_i| (the usual backward analysis of the ratio recurrence: the ratio of two
// carried minors obeys it with the step's rounding factors folded into d_i and e_{i-1}^2), so on the
// scaled T (|d_i|, |e_i|, |x| <= 1) ||T' - T|| <= 7u. A count of c at x thus brackets: the exact
// counts at x - 7u and x + 7u lie below and above c.
__device__ __forceinline__ int sturm_count_f32(const float* __restrict__ d, const float* __restrict__ e2, int n,
                                               float x) {
  float a0 = 1.0f, a1 = d[0] - x;
  if (a1 == 0.0f) a1 = -0x1p-60f;
  int cnt = a1 < 0.0f;
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    float t = fmaf(d[i] - x, a1, -e2[i - 1] * a0);
    const unsigned ex = (__float_as_uint(t) >> 23) & 0xFFu;
    if (ex - (127u - 40u) > 80u) {  // exponent outside [-40, 40], zero or subnormal
      if (t == 0.0f) t = -0x1p-60f * a1;
      const float f = fabsf(t) > 1.0f ? 0x1p-40f : 0x1p+40f;
      if (fabsf(t) > 0x1p+40f || fabsf(t) < 0x1p-40f) {
        t *= f;
        a1 *= f;
      }
    }
    cnt += (__float_as_int(t) ^ __float_as_int(a1)) < 0;
    a0 = a1;
    a1 = t;
  }
  return cnt;
}

// L lanes share an eigenvalue and evaluate L interior points of its interval
// per round (multisection): the interval shrinks (L + 1)-fold per round. The
// first rounds count in FP32 until the interval is 2^-17 ||T|| wide; it is then
// widened by 2^-18 ||T|| (over nine times the FP32 counts' error bound, see
// sturm_count_f32) and the FP64 rounds take over. An interval stops at a width of
// 2 eps |lambda| or 4 eps ||T||: the tridiagonalisation already perturbs every
// eigenvalue by about eps ||T||.
template <int L>
__global__ void __launch_bounds__(128) bisect_kernel(const double* __restrict__ dg, const double* __restrict__ eg,
                                                     int n, double* __restrict__ lam, int j0, int j1) {
  extern __shared__ double tsm[];
  double* d = tsm;       // scaled diagonal
  double* e2 = tsm + n;  // scaled squared off-diagonal
  float* d32 = reinterpret_cast<float*>(tsm + 2 * (size_t)n);  // the same in FP32
  float* e32 = d32 + n;
  __shared__ double red_lo[4], red_hi[4];
  // Gershgorin interval of T, block-wide
  double gl = INFINITY, gu = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = (i > 0 ? fabs(eg[i - 1]) : 0.0) + (i + 1 < n ? fabs(eg[i]) : 0.0);
    gl = fmin(gl, dg[i] - r);
    gu = fmax(gu, dg[i] + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red_lo[threadIdx.x >> 5] = gl;
    red_hi[threadIdx.x >> 5] = gu;
  }
  __syncthreads();
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {  // 1, 2 or 4 warps
    gl = fmin(gl, red_lo[w]);
    gu = fmax(gu, red_hi[w]);
  }
  const double tnorm = fmax(fmax(fabs(gl), fabs(gu)), DBL_MIN);
  int ex = 0;
  frexp(tnorm, &ex);
  const double sc = ldexp(1.0, -ex);  // tnorm * sc in [0.5, 1)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = dg[i] * sc;
    const double ei = (i + 1 < n) ? eg[i] * sc : 0.0;
    e2[i] = ei * ei;
    d32[i] = (float)d[i];
    e32[i] = (float)e2[i];
  }
  __syncthreads();
  const int sub = (threadIdx.x & 31) / L;                   // eigenvalue slot in the warp
  const int g = threadIdx.x & (L - 1);                      // point of the multisection
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int j = j0 + warp_global * (32 / L) + sub;          // descending index
  const int k = n - 1 - j;                                  // ascending index
  const bool active = j < j1;
  const double tn = tnorm * sc;
  const double abs_floor = 4.0 * DBL_EPSILON * tn;
  double lo = gl * sc - 2.0 * DBL_EPSILON * tn * n, hi = gu * sc + 2.0 * DBL_EPSILON * tn * n;
  const unsigned gmask = (0xffffffffu >> (32 - L)) << (sub * L);
  // FP32 rounds down to a width of 2^-17 (tn is in [0.5, 1)); an interval they moved is widened after
  bool moved = false;
  for (int it = 0; it < 16; ++it) {
    const bool done = !active || hi - lo <= 0x1p-17;
    if (__all_sync(0xffffffffu, done)) break;
    const double step = (hi - lo) / (double)(L + 1);
    const double x = lo + step * (double)(g + 1);
    const bool above = !done && sturm_count_f32(d32, e32, n, (float)x) > k;
    const unsigned bal = __ballot_sync(0xffffffffu, above) & gmask;
    if (!done) {
      const unsigned mine = bal >> (sub * L);
      const int first = mine ? __ffs(mine) - 1 : L;
      const double nlo = (first == 0) ? lo : lo + step * (double)first;
      const double nhi = (first == L) ? hi : lo + step * (double)(first + 1);
      lo = nlo;
      hi = nhi;
      moved = true;
    }
  }
  if (moved) {
    lo -= 0x1p-18;
    hi += 0x1p-18;
  }
  for (int it = 0; it < 64; ++it) {
    const bool done = !active || hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + abs_floor;
    if (__all_sync(0xffffffffu, done)) break;
    const double step = (hi - lo) / (double)(L + 1);
    const double x = lo + step * (double)(g + 1);
    const bool above = !done && sturm_count(d, e2, n, x) > k;
    const unsigned bal = __ballot_sync(0xffffffffu, above) & gmask;
    if (!done) {
      // counts grow with x, so the points above eigenvalue k form a suffix
      const unsigned mine = bal >> (sub * L);
      const int first = mine ? __ffs(mine) - 1 : L;  // first point above
      const double nlo = (first == 0) ? lo : lo + step * (double)first;
      const double nhi = (first == L) ? hi : lo + step * (double)(first + 1);
      lo = nlo;
      hi = nhi;
    }
  }
  if (active && g == 0) lam[j] = 0.5 * (lo + hi) / sc;
}

// ---------------------------------------------------------------------------
// Eigenvectors of T for the r largest eigenvalues by twisted factorisation:
// with the stationary (top-down) and progressive (bottom-up) LDL^T
// factorisations of T - lambda I, the twist index k minimising
// |gamma_k| = |D+_k + D-_k - (d_k - lambda)| gives the eigenvector from
// z_k = 1 and two one-sided recurrences. One lane per eigenvalue; inside a
// chain of numerically equal eigenvalues (gaps within 10 eps ||T||) the
// shifts are spread by 10 eps ||T|| per member so the members differ, and
// cluster_orth_kernel then orthogonalises each cluster (a chain of
// eigenvalues closer than ctol = 1e-9 ||T||).
// Z[i * r + j] receives component i of eigenvector j of T.
// Scratch: 4 n r doubles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double cluster_tol(const double* lam, int n) {
  return 1e-9 * (fmax(fabs(lam[0]), fabs(lam[n - 1])) + DBL_MIN);
}

__global__ void __launch_bounds__(64) invit_kernel(const double* dg, const double* eg, int n,
                                                   const double* __restrict__ lam, int r, double* __restrict__ Z,
                                                   double* __restrict__ scratch) {
  // 32 eigenvalues per CTA, lane = eigenvalue; warp 0 runs the forward factorisation and the
  // recurrence below the twist, warp 1 the backward factorisation and the recurrence above it (the
  // two halves of each step are independent chains of FP64 divisions and products)
  extern __shared__ double tsm[];
  __shared__ double bestv[2][32], part[2][32];
  __shared__ int bestk[2][32];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    tsm[i] = dg[i];
    tsm[n + i] = eg[i];
  }
  __syncthreads();
  const double* d = tsm;
  const double* e = tsm + n;
  const int lane = threadIdx.x & 31, half = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  const bool act = j < r;
  const double tnorm = fmax(fabs(lam[0]), fabs(lam[n - 1])) + DBL_MIN;
  const double tiny = 1e-3 * DBL_EPSILON * tnorm + DBL_MIN;
  // scratch [4][n][r]: D+, L+, D-, U- with the eigenvalue index innermost (coalesced per step)
  const int64_t R = r;
  double* Dp = scratch + j;
  double* Lp = scratch + (int64_t)n * R + j;
  double* Dm = scratch + 2 * (int64_t)n * R + j;
  double* Um = scratch + 3 * (int64_t)n * R + j;
  double s = 0.0;
  if (act) {
    // the shift offset counts members of the chain of numerically equal eigenvalues only (gaps within
    // 10 eps ||T||): spread over a whole 1e-9 ||T|| chain it would grow past the local gaps and move
    // later members onto their neighbours' eigenvalues
    const double etol = 10.0 * DBL_EPSILON * tnorm;
    int lead = j;
    while (lead > 0 && fabs(lam[lead - 1] - lam[lead]) <= etol) --lead;
    s = lam[j] + (double)(j - lead) * etol;
    if (half == 0) {
      double dp = d[0] - s;
      for (int i = 0; i + 1 < n; ++i) {
        if (fabs(dp) < tiny) dp = tiny;
        const double l = e[i] / dp;
        Dp[(int64_t)i * R] = dp;
        Lp[(int64_t)i * R] = l;
        dp = (d[i + 1] - s) - l * e[i];
      }
      Dp[(int64_t)(n - 1) * R] = dp;
    } else {
      double dm = d[n - 1] - s;
      for (int i = n - 1; i >= 1; --i) {
        if (fabs(dm) < tiny) dm = tiny;
        const double u = e[i - 1] / dm;
        Dm[(int64_t)i * R] = dm;
        Um[(int64_t)i * R] = u;
        dm = (d[i - 1] - s) - u * e[i - 1];
      }
      Dm[0] = dm;
    }
  }
  __syncthreads();
  // twist index: the first i of least |D+_i + D-_i - (d_i - s)|, each warp over half of the range
  const int mid = n / 2;
  {
    int k = 0;
    double best = INFINITY;
    if (act) {
      const int lo = half == 0 ? 0 : mid, hi = half == 0 ? mid : n;
      for (int i = lo; i < hi; ++i) {
        const double g = fabs(Dp[(int64_t)i * R] + Dm[(int64_t)i * R] - (d[i] - s));
        if (g < best) {
          best = g;
          k = i;
        }
      }
    }
    bestv[half][lane] = best;
    bestk[half][lane] = k;
  }
  __syncthreads();
  const int k = (bestv[1][lane] < bestv[0][lane]) ? bestk[1][lane] : bestk[0][lane];
  // z in the output column: z_k = 1, then the two one-sided recurrences
  double* zc = Z + j;
  double mx = 1.0;
  if (act) {
    if (half == 0) {
      zc[(int64_t)k * R] = 1.0;
      double z = 1.0;
      for (int i = k - 1; i >= 0; --i) {
        z = -Lp[(int64_t)i * R] * z;
        zc[(int64_t)i * R] = z;
        mx = fmax(mx, fabs(z));
      }
    } else {
      double z = 1.0;
      for (int i = k + 1; i < n; ++i) {
        z = -Um[(int64_t)i * R] * z;
        zc[(int64_t)i * R] = z;
        mx = fmax(mx, fabs(z));
      }
    }
  }
  part[half][lane] = mx;
  __syncthreads();
  mx = fmax(part[0][lane], part[1][lane]);
  if (!isfinite(mx)) mx = 1.0;
  const double inv_mx = 1.0 / mx;
  __syncthreads();
  double nrm = 0.0;
  const int lo = half == 0 ? 0 : mid, hi = half == 0 ? mid : n;
  if (act)
    for (int i = lo; i < hi; ++i) {
      const double z = zc[(int64_t)i * R] * inv_mx;
      nrm = fma(z, z, nrm);
    }
  part[half][lane] = nrm;
  __syncthreads();
  nrm = part[0][lane] + part[1][lane];
  const double sc = nrm > 0.0 ? inv_mx / sqrt(nrm) : 0.0;
  if (act)
    for (int i = lo; i < hi; ++i) zc[(int64_t)i * R] *= sc;
}

// One CTA per potential cluster leader j < r (an index that starts a chain of
// at least two eigenvalues closer than ctol, chains cut at r): classical
// Gram-Schmidt of every later member against the earlier ones, twice, then
// normalisation. Dot products one warp per earlier member; the update one
// thread per component.
__global__ void __launch_bounds__(EIG_THREADS) cluster_orth_kernel(const double* __restrict__ lam, int n, int r,
                                                                   double* __restrict__ Z) {
  const int j0 = blockIdx.x;
  const double ctol = cluster_tol(lam, n);
  if (j0 + 1 >= r || fabs(lam[j0] - lam[j0 + 1]) > ctol) return;
  if (j0 > 0 && fabs(lam[j0 - 1] - lam[j0]) <= ctol) return;  // not the leader
  int cs = 2;
  while (j0 + cs < r && fabs(lam[j0 + cs - 1] - lam[j0 + cs]) <= ctol) ++cs;
  extern __shared__ double dots[];  // cs
  __shared__ double red[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = j0 + 1; m < j0 + cs; ++m) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int q = j0 + warp; q < m; q += nw) {
        double dt = 0.0;
        for (int i = lane; i < n; i += 32) dt = fma(Z[(int64_t)i * r + q], Z[(int64_t)i * r + m], dt);
        dt = warp_sum(dt);
        if (lane == 0) dots[q - j0] = dt;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double* row = Z + (int64_t)i * r;
        double acc = row[m];
        for (int q = j0; q < m; ++q) acc = fma(-dots[q - j0], row[q], acc);
        Z[(int64_t)i * r + m] = acc;
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s2 = fma(Z[(int64_t)i * r + m], Z[(int64_t)i * r + m], s2);
    const double nrm = block_sum(s2, red);
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Z[(int64_t)i * r + m] *= inv;
    __syncthreads();
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct WorkLayout {
  double *Vh, *d, *e, *tau, *pbuf, *pub;
  Barrier* bar;
};

WorkLayout layout(void* work, int64_t n) {
  char* p = static_cast<char*>(work);
  WorkLayout L;
  L.Vh = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * n * n);
  L.d = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * n);
  L.e = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * n);
  L.tau = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * n);
  L.pbuf = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * 2 * n);
  L.pub = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * 2 * n);
  L.bar = reinterpret_cast<Barrier*>(p);
  return L;
}

}  // namespace

size_t eig_workspace_bytes(int64_t n) {
  return align256(sizeof(double) * n * n) + 3 * align256(sizeof(double) * n) + 2 * align256(sizeof(double) * 2 * n) +
         256;
}

size_t eig_vectors_scratch_bytes(int64_t n, int64_t r) {
  return std::max(sizeof(double) * 4 * (size_t)n * (size_t)r + 256, wy_workspace_bytes(n));
}

// ---------------------------------------------------------------------------
// Autotuned shape of the resident-rows tridiagonalisation. Rows per CTA trade the FP64 work each SM
// does per column (fewer rows: more SMs share it) against the width of the grid barrier and the
// occupancy (one or two CTAs per SM). The first matrix of each size bucket (32 rows wide) runs every
// candidate that fits, timed with CUDA events on the launching stream, and the fastest is kept for the
// bucket in this process; the candidates compute the same reduction, so any run's output is valid.
// Off unless BHT_AUTOTUNE=1: timed alone the tuned shapes are a few per cent faster, but they take SMs
// that the other nodes of a layer, solved at the same time on their own streams, then wait for. The
// fixed rule (at least eight rows, at most one CTA per SM) leaves those SMs free.
// ---------------------------------------------------------------------------
namespace {
// Test hook of the timeout path: the next g_withhold cooperative tridiagonalisations with more than
// one CTA run with CTA 0 withholding its first grid-barrier arrival and a wait limit of g_wait_ms.
std::atomic<int> g_withhold{0};
std::atomic<int> g_wait_ms{0};

unsigned int take_barrier_test_flags() {
  int n = g_withhold.load();
  while (n > 0 && !g_withhold.compare_exchange_weak(n, n - 1)) {
  }
  if (n <= 0) return 0u;
  const unsigned int ms = (unsigned int)std::min(std::max(g_wait_ms.load(), 1), 65535);
  return 1u | (ms << 16);
}

__global__ void set_barrier_flags_kernel(Barrier* bar, unsigned int flags) { bar->flags = flags; }

// Before a multi-CTA launch of the resident-rows tridiagonalisation (its barrier word already cleared).
cudaError_t arm_barrier_test(Barrier* bar, cudaStream_t s) {
  const unsigned int flags = take_barrier_test_flags();
  if (!flags) return cudaSuccess;
  set_barrier_flags_kernel<<<1, 1, 0, s>>>(bar, flags);
  note_launch();
  return cudaGetLastError();
}

std::mutex g_tune_mu;
std::vector<std::pair<int64_t, int>> g_tune;  // (device * 4096 + bucket, rows per CTA)

bool autotune_on() {
  static const bool on = [] {
    const char* v = std::getenv("BHT_AUTOTUNE");
    return v && v[0] == '1';
  }();
  return on;
}

int tuned_rows(int64_t key) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& t : g_tune)
    if (t.first == key) return t.second;
  return -1;
}

void remember_rows(int64_t key, int rpb) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto& t : g_tune)
    if (t.first == key) {
      t.second = rpb;
      return;
    }
  g_tune.push_back({key, rpb});
}

// One launch of the resident-rows kernel with rpb rows per CTA (the barrier word is cleared first);
// cudaErrorInvalidConfiguration when the shape does not fit (shared memory or co-residency).
cudaError_t launch_rows(const double* G, int n, int rpb, const WorkLayout& L, int* status, int nsm, cudaStream_t s) {
  const int nbk = (n + rpb - 1) / rpb;
  const size_t smr = sizeof(double) * (size_t)(rpb + 4) * (size_t)n;
  if (smr > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(tridiag_rows_kernel));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.bar, 0, sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  if (nbk > 1) {
    e = arm_barrier_test(L.bar, s);
    if (e != cudaSuccess) return e;
  }
  int nn = n, r = rpb;
  const double* Gc = G;
  double *Vh = L.Vh, *d = L.d, *ee = L.e, *tau = L.tau, *pbuf = L.pbuf, *pub = L.pub;
  Barrier* bar = L.bar;
  if (nbk == 1) {
    tridiag_rows_kernel<<<1, EIG_THREADS, smr, s>>>(Gc, nn, r, Vh, d, ee, tau, pbuf, pub, bar, status);
    note_launch();
    return cudaGetLastError();
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_rows_kernel, EIG_THREADS, smr);
  if (e != cudaSuccess) return e;
  if ((int64_t)per_sm * nsm < nbk) return cudaErrorInvalidConfiguration;
  void* args[] = {&Gc, &nn, &r, &Vh, &d, &ee, &tau, &pbuf, &pub, &bar, &status};
  e = cudaLaunchCooperativeKernel((void*)tridiag_rows_kernel, dim3(nbk), dim3(EIG_THREADS), args, smr, s);
  note_launch();
  return e;
}

// Time the candidates on G and return the fastest rows per CTA (the last run leaves a valid output).
int tune_rows(const double* G, int n, const WorkLayout& L, int* status, int nsm, cudaStream_t s) {
  const int warps = EIG_THREADS / 32;
  std::vector<int> cand = {(n + nsm - 1) / nsm, (n + 2 * nsm - 1) / (2 * nsm), warps / 2, warps, 2 * warps};
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  int best = -1;
  float best_ms = 0.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1;
  }
  for (int rpb : cand) {
    if (rpb < 1 || rpb > n) continue;
    cudaEventRecord(e0, s);
    if (launch_rows(G, n, rpb, L, status, nsm, s) != cudaSuccess) {
      cudaGetLastError();  // a shape that does not fit is simply not a candidate
      continue;
    }
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    if (best < 0 || ms < best_ms) {
      best = rpb;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}
}  // namespace

cudaError_t launch_eig_tridiag(double* G, int64_t n, void* work, int* status, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (n > 4096) return cudaErrorInvalidValue;
  WorkLayout L = layout(work, n);
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(Barrier), s);
  if (e != cudaSuccess) return e;
  const size_t sm = 2 * sizeof(double) * (size_t)n;
  if (sm > 0) {  // dynamic + static must fit the cap
    e = allow_max_smem(reinterpret_cast<const void*>(tridiag_kernel));
    if (e != cudaSuccess) return e;
  }
  const double flops = 4.0 / 3.0 * (double)n * (double)n * (double)n;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (n > ONE_CTA_N && autotune_on()) {
    const int64_t key = (int64_t)dev * 4096 + (n + 31) / 32;
    int rpb = tuned_rows(key);
    if (rpb < 0) {
      ProfScope prof(K_EIG_TRIDIAG, s, flops, 16.0 * (double)n * (double)n);
      rpb = tune_rows(G, (int)n, L, status, nsm, s);
      if (rpb > 0) {
        remember_rows(key, rpb);
        return cudaSuccess;  // the last candidate's output stands
      }
    } else {
      ProfScope prof(K_EIG_TRIDIAG, s, flops, 16.0 * (double)n * (double)n);
      if (launch_rows(G, (int)n, std::min<int>(rpb, (int)n), L, status, nsm, s) == cudaSuccess) return cudaSuccess;
      cudaGetLastError();  // fall through to the fixed rule
    }
  }
  if (n >= 3) {
    // rows resident in shared memory: one CTA for a small matrix, else about one warp per row
    // (at least ceil(n / #SM) rows per CTA, at most one CTA per SM)
    const int warps = EIG_THREADS / 32;
    const int rpb = n <= ONE_CTA_N ? (int)n : (int)std::max<int64_t>(warps, (n + nsm - 1) / nsm);
    const int nbk = (int)((n + rpb - 1) / rpb);
    const size_t smr = sizeof(double) * (size_t)(rpb + 4) * (size_t)n;
    if (smr <= 200 * 1024) {
      if (smr > 0) {  // dynamic + static must fit the cap
        e = allow_max_smem(reinterpret_cast<const void*>(tridiag_rows_kernel));
        if (e != cudaSuccess) return e;
      }
      ProfScope prof(K_EIG_TRIDIAG, s, flops, 16.0 * (double)n * (double)n);
      int nn = (int)n, r = rpb;
      const double* Gc = G;
      if (nbk == 1) {
        tridiag_rows_kernel<<<1, EIG_THREADS, smr, s>>>(Gc, nn, r, L.Vh, L.d, L.e, L.tau, L.pbuf, L.pub, L.bar,
                                                         status);
        note_launch();
        return cudaGetLastError();
      }
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_rows_kernel, EIG_THREADS, smr);
      if (e != cudaSuccess) return e;
      if ((int64_t)per_sm * nsm >= nbk) {
        e = arm_barrier_test(L.bar, s);
        if (e != cudaSuccess) return e;
        void* args[] = {&Gc, &nn, &r, &L.Vh, &L.d, &L.e, &L.tau, &L.pbuf, &L.pub, &L.bar, &status};
        e = cudaLaunchCooperativeKernel((void*)tridiag_rows_kernel, dim3(nbk), dim3(EIG_THREADS), args, smr, s);
        note_launch();
        return e;
      }
    }
  }
  if (n <= SMALL_N) {
    ProfScope prof(K_EIG_TRIDIAG, s, flops, 16.0 * (double)n * (double)n);
    tridiag_kernel<<<1, EIG_THREADS, sm, s>>>(G, (int)n, L.Vh, L.d, L.e, L.tau, L.pbuf, L.bar, status);
    note_launch();
    return cudaGetLastError();
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_kernel, EIG_THREADS, sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // about one warp per row, never more CTAs than can be co-resident
  const int64_t want = (n + (EIG_THREADS / 32) - 1) / (EIG_THREADS / 32);
  const int blocks = (int)std::min<int64_t>(want, (int64_t)nsm * std::min(per_sm, 2));
  int nn = (int)n;
  void* args[] = {&G, &nn, &L.Vh, &L.d, &L.e, &L.tau, &L.pbuf, &L.bar, &status};
  ProfScope prof(K_EIG_TRIDIAG, s, flops, 16.0 * (double)n * (double)n);
  e = cudaLaunchCooperativeKernel((void*)tridiag_kernel, dim3(blocks), dim3(EIG_THREADS), args, sm, s);
  note_launch();
  return e;
}

template <int L>
cudaError_t launch_bisect_l(int64_t n, const double* d, const double* e, double* lam, int64_t j0, int64_t j1,
                            cudaStream_t s) {
  const size_t sm = (2 * sizeof(double) + 2 * sizeof(float)) * (size_t)n;
  if (sm > 0) {  // dynamic + static must fit the cap
    cudaError_t e2 = allow_max_smem(reinterpret_cast<const void*>(bisect_kernel<L>));
    if (e2 != cudaSuccess) return e2;
  }
  // CTAs of 128, 64 or 32 threads: the largest that still gives every SM a CTA (the Sturm sequences are
  // FP64 dependency chains, so the eigenvalues are best spread over all SMs)
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t threads = (j1 - j0) * L;
  int bs = 128;
  while (bs > 32 && threads / bs < nsm) bs >>= 1;
  const int64_t per_block = bs / L;  // eigenvalues per CTA
  const int64_t blocks = (j1 - j0 + per_block - 1) / per_block;
  // algorithmic work: 3 FP64 operations per Sturm step, about 53 / log2(L + 1) rounds of L points
  ProfScope prof(K_EIG_BISECT, s, 3.0 * (double)n * (double)L * (53.0 / std::log2((double)L + 1.0)) * (double)(j1 - j0),
                 16.0 * (double)n);
  bisect_kernel<L><<<(unsigned)blocks, bs, sm, s>>>(d, e, (int)n, lam, (int)j0, (int)j1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_eig_bisect(int64_t n, void* work, double* lam, int64_t j0, int64_t j1, cudaStream_t s) {
  if (n <= 0 || j1 <= j0) return cudaSuccess;
  WorkLayout L = layout(work, n);
  // 16 points per eigenvalue once there are enough eigenvalues to give every SM sub-partition a warp,
  // 32 below that (fewer rounds)
  if (j1 - j0 >= 512) return launch_bisect_l<16>(n, L.d, L.e, lam, j0, j1, s);
  return launch_bisect_l<32>(n, L.d, L.e, lam, j0, j1, s);
}

const double* eig_tridiag_diagonal(void* work, int64_t n) { return layout(work, n).d; }

cudaError_t launch_eig_values(double* G, int64_t n, double* lam, void* work, int* status, cudaStream_t s) {
  cudaError_t e = launch_eig_tridiag(G, n, work, status, s);
  if (e != cudaSuccess) return e;
  return launch_eig_bisect(n, work, lam, 0, n, s);
}

cudaError_t launch_eig_vectors(int64_t n, int64_t r, const double* lam, double* U, void* work, void* scratch,
                               cudaStream_t s) {
  if (n <= 0 || r <= 0) return cudaSuccess;
  WorkLayout L = layout(work, n);
  {
    ProfScope prof(K_EIG_INVIT, s);
    const size_t sm = 2 * sizeof(double) * (size_t)n;
    if (sm > 0) {  // dynamic + static must fit the cap
      cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(invit_kernel));
      if (e != cudaSuccess) return e;
    }
    invit_kernel<<<(unsigned)((r + 31) / 32), 64, sm, s>>>(L.d, L.e, (int)n, lam, (int)r, U,
                                                           static_cast<double*>(scratch));
    note_launch();
    if (r >= 2) {
      // every index may lead a cluster; a cluster never exceeds r members
      const size_t smc = sizeof(double) * (size_t)r;
      if (smc > 0) {  // dynamic + static must fit the cap
        cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(cluster_orth_kernel));
        if (e != cudaSuccess) return e;
      }
      cluster_orth_kernel<<<(unsigned)r, EIG_THREADS, smc, s>>>(lam, (int)n, (int)r, U);
      note_launch();
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (n >= 3) {
    // U = H_0 H_1 ... H_{n-3} Z in blocks of reflectors (compact WY form, wy.cu); the block factors go to
    // the scratch space, which the inverse iteration no longer needs
    ProfScope prof(K_EIG_BACK, s, 2.0 * (double)n * (double)n * (double)r,
                   8.0 * (double)n * (0.5 * (double)n + 2.0 * (double)r));
    e = launch_wy_apply(L.Vh, n, 1, 1, L.tau, n - 2, n, U, r, 0, r, U, r, scratch, s);
  }
  return e;
}

}  // namespace bht

extern "C" bht_status bht_debug_withhold_barrier(int32_t launches, int32_t wait_ms) {
  if (launches < 0 || wait_ms < 1 || wait_ms > 65535) {
    bht::set_last_error("launches >= 0 and 1 <= wait_ms <= 65535");
    return BHT_EINVAL;
  }
  bht::g_wait_ms.store(wait_ms);
  bht::g_withhold.store(launches);
  return BHT_OK;
}

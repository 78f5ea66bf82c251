// mlp.cu — the rank / expansion predictor: a three-layer perceptron (66 -> 128 -> 128 -> 2) with
// bf16 weights and activations and FP32 accumulation, its loss, gradients and Adam step, and the
// sketched singular-value features of a node's residual Gram matrix that it reads.
//
// Forward (per sample x): x~ = bf16(x); a1 = bf16(W1) x~ + b1; h1 = bf16(relu(a1));
// a2 = bf16(W2) h1 + b2; h2 = bf16(relu(a2)); o = bf16(W3) h2 + b3. o0 is the predicted rank as a
// fraction of the node's largest possible rank, o1 the logit of "the batch expands this node".
// Loss: mean over the batch of (o0 - t0)^2 + log(1 + exp(o1)) - t1 o1. Gradients are taken with
// respect to the rounded weights in the arithmetic of the forward pass and applied to an FP32
// master copy by Adam. Parameters are flattened as W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// W3 [2][H], b3 [2].
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace bht {

namespace {

constexpr int MT = 256;

// out[b][j] = sum_i W[j][i] in[b][i] + bias[j] (FP32 accumulation); pre-activation to `pre`
// (nullable), then relu and bf16 rounding when `hidden`.
__global__ void linear_fwd_kernel(const __nv_bfloat16* __restrict__ in, int64_t B, int nin,
                                  const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias, int nout,
                                  float* __restrict__ pre, __nv_bfloat16* __restrict__ act, float* __restrict__ out) {
  const int64_t total = B * nout;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / nout;
    const int j = (int)(e - b * nout);
    const __nv_bfloat16* x = in + b * nin;
    const __nv_bfloat16* w = W + (int64_t)j * nin;
    float acc = 0.f;
    for (int i = 0; i < nin; ++i) acc = fmaf(__bfloat162float(w[i]), __bfloat162float(x[i]), acc);
    acc += bias[j];
    if (pre) pre[e] = acc;
    if (act) act[e] = __float2bfloat16_rn(fmaxf(acc, 0.f));
    if (out) out[e] = acc;
  }
}

__global__ void round_input_kernel(const float* __restrict__ X, int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(X[e]);
}

// dO = d loss / d o for the mean loss; loss summed in FP64.
__global__ void loss_kernel(const float* __restrict__ o, const float* __restrict__ T, int64_t B,
                            float* __restrict__ dO, double* __restrict__ loss) {
  double part = 0.0;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (int64_t)gridDim.x * blockDim.x) {
    const float o0 = o[2 * b], o1 = o[2 * b + 1], t0 = T[2 * b], t1 = T[2 * b + 1];
    const float d0 = o0 - t0;
    // log(1 + exp(o1)) evaluated without overflow
    const float sp = fmaxf(o1, 0.f) + log1pf(expf(-fabsf(o1)));
    part += (double)(d0 * d0) + (double)(sp - t1 * o1);
    const float sig = 1.f / (1.f + expf(-o1));
    dO[2 * b] = 2.f * d0 / (float)B;
    dO[2 * b + 1] = (sig - t1) / (float)B;
  }
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) part += __shfl_xor_sync(0xffffffffu, part, k);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / (double)B);
}

// G[r][c] = sum_b A[b][r] Bm[b][c]: the weight gradient of a layer (A: output gradients [B][R],
// Bm: the layer's bf16 inputs [B][C]); also gb[r] = sum_b A[b][r] when gb is not null.
__global__ void outer_reduce_kernel(const float* __restrict__ A, int64_t B, int R, const __nv_bfloat16* __restrict__ Bm,
                                    int C, float* __restrict__ G, float* __restrict__ gb) {
  const int64_t total = (int64_t)R * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / C), c = (int)(e - (int64_t)r * C);
    float acc = 0.f;
    for (int64_t b = 0; b < B; ++b) acc = fmaf(A[b * R + r], __bfloat162float(Bm[b * C + c]), acc);
    G[e] = acc;
    if (gb && c == 0) {
      float s = 0.f;
      for (int64_t b = 0; b < B; ++b) s += A[b * R + r];
      gb[r] = s;
    }
  }
}

// D[b][i] = (sum_j dA[b][j] W[j][i]) * (pre[b][i] > 0): the gradient at the previous layer's
// pre-activation (W: bf16 [J][I]).
__global__ void backprop_kernel(const float* __restrict__ dA, int64_t B, int J, const __nv_bfloat16* __restrict__ W,
                                int I, const float* __restrict__ pre, float* __restrict__ D) {
  const int64_t total = B * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / I;
    const int i = (int)(e - b * I);
    float acc = 0.f;
    for (int j = 0; j < J; ++j) acc = fmaf(dA[b * J + j], __bfloat162float(W[(int64_t)j * I + i]), acc);
    D[e] = pre[e] > 0.f ? acc : 0.f;
  }
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float c1, float c2, float beta1,
                            float beta2, float eps) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = beta1 * m[e] + (1.f - beta1) * ge;
    const float ve = beta2 * v[e] + (1.f - beta2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    w[e] -= lr * (me * c1) / (sqrtf(ve * c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, int64_t n, __nv_bfloat16* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(w[e]);
}

int grid1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + MT - 1) / MT, 152 * 8)); }

// ---------------------------------------------------------------------------
// Sketch features. For a symmetric positive semidefinite Gram matrix G (c x c, FP64) of a node
// unfolding M (G = M M^T), S = Omega^T G Omega = (Omega^T M)(Omega^T M)^T is the Gram matrix of
// a Gaussian sketch of width k of M (Omega c x k, entries N(0, 1/k) from a counter-based hash and
// the Box-Muller transform). Its eigenvalues are the squared singular values of the sketch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Omega [c][k], N(0, 1/k)
__global__ void gauss_sketch_kernel(float* __restrict__ Om, int64_t c, int k, uint64_t seed) {
  const int64_t total = c * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = mix64(seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1));
    const float u1 = ((float)(z >> 40) + 0.5f) * 0x1.0p-24f;  // (0, 1)
    const float u2 = (float)((z >> 16) & 0xFFFFFF) * 0x1.0p-24f;
    Om[e] = sqrtf(-2.f * logf(u1)) * cospif(2.f * u2) * rsqrtf((float)k);
  }
}

// T [k][c] = Omega^T G (FP32 accumulation of the FP64 Gram rounded to FP32)
__global__ void sketch_left_kernel(const double* __restrict__ G, int64_t c, const float* __restrict__ Om, int k,
                                   float* __restrict__ T) {
  const int64_t total = (int64_t)k * c;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / c);
    const int64_t j = e - (int64_t)q * c;
    float acc = 0.f;
    for (int64_t i = 0; i < c; ++i) acc = fmaf(Om[i * k + q], (float)G[i * c + j], acc);
    T[e] = acc;
  }
}

// S [k][k] = T Omega
__global__ void sketch_right_kernel(const float* __restrict__ T, int64_t c, const float* __restrict__ Om, int k,
                                    float* __restrict__ S) {
  const int total = k * k;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int p = e / k, q = e - p * k;
    float acc = 0.f;
    for (int64_t j = 0; j < c; ++j) acc = fmaf(T[(int64_t)p * c + j], Om[j * k + q], acc);
    S[e] = acc;
  }
}

// Eigenvalues of the symmetric S (n x n, n <= 128, FP32) by cyclic Jacobi in one CTA with the
// matrix in shared memory: each round rotates n/2 disjoint pairs (round-robin ordering); sweeps
// stop when the off-diagonal mass is below 1e-7 of the diagonal's or after 12 sweeps. Then the
// features: f[i] = log10(s_i / s_1) for the descending singular values s_i = sqrt(max(lambda_i, 0))
// of the sketch (-16 below s_1 * 1e-16 or past the sketch), i < 64; f[64] = log10(tol / ||M||)
// with ||M||^2 read from norm2 (device); f[65] = log2(c) / 10.
__global__ void __launch_bounds__(256) jacobi_features_kernel(const float* __restrict__ S, int n, double tol,
                                                              const double* __restrict__ norm2, int64_t c,
                                                              float* __restrict__ f) {
  extern __shared__ float a[];  // n x n, then n eigenvalues
  __shared__ int pairs[2][64];
  __shared__ float cs[64], sn[64];
  __shared__ float red[32];
  float* lam = a + n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) a[e] = S[e];
  __syncthreads();
  const int m = (n + 1) / 2 * 2;  // even number of players (one dummy when n is odd)
  for (int sweep = 0; sweep < 12; ++sweep) {
    // convergence: off-diagonal vs diagonal mass
    float off = 0.f, dia = 0.f;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      if (i == j) dia += a[e] * a[e]; else off += a[e] * a[e];
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, k);
      dia += __shfl_xor_sync(0xffffffffu, dia, k);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = off;
      red[16 + (threadIdx.x >> 5)] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float o = 0.f, d = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        o += red[w];
        d += red[16 + w];
      }
      red[0] = (o <= 1e-14f * d) ? 1.f : 0.f;
    }
    __syncthreads();
    const bool done = red[0] != 0.f;
    __syncthreads();
    if (done) break;
    for (int round = 0; round < m - 1; ++round) {
      // round-robin pairing: player 0 fixed, the others rotate
      if (threadIdx.x < m / 2) {
        const int t = threadIdx.x;
        int p = (t == 0) ? 0 : 1 + (t - 1 + round) % (m - 1);
        int q = 1 + (m - 2 - t + round) % (m - 1);
        if (p > q) { const int x = p; p = q; q = x; }
        pairs[0][t] = p;
        pairs[1][t] = q;
      }
      __syncthreads();
      // rotation angles, one thread per pair (stored in the pair slot)
      if (threadIdx.x < m / 2) {
        const int p = pairs[0][threadIdx.x], q = pairs[1][threadIdx.x];
        float c_ = 1.f, s_ = 0.f;
        if (q < n && p < n) {
          const float apq = a[p * n + q];
          if (apq != 0.f) {
            const float theta = (a[q * n + q] - a[p * n + p]) / (2.f * apq);
            const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            c_ = rsqrtf(t * t + 1.f);
            s_ = t * c_;
          }
        }
        cs[threadIdx.x] = c_;
        sn[threadIdx.x] = s_;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = threadIdx.x; e < (m / 2) * n; e += blockDim.x) {
        const int t = e / n, j = e - t * n;
        const int p = pairs[0][t], q = pairs[1][t];
        if (q >= n) continue;
        const float ap = a[p * n + j], aq = a[q * n + j];
        a[p * n + j] = cs[t] * ap - sn[t] * aq;
        a[q * n + j] = sn[t] * ap + cs[t] * aq;
      }
      __syncthreads();
      // columns: A <- A J
      for (int e = threadIdx.x; e < (m / 2) * n; e += blockDim.x) {
        const int t = e / n, i = e - t * n;
        const int p = pairs[0][t], q = pairs[1][t];
        if (q >= n) continue;
        const float ap = a[i * n + p], aq = a[i * n + q];
        a[i * n + p] = cs[t] * ap - sn[t] * aq;
        a[i * n + q] = sn[t] * ap + cs[t] * aq;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = fmaxf(a[i * n + i], 0.f);
  __syncthreads();
  if (threadIdx.x == 0) {
    // descending order (insertion sort, n <= 128)
    for (int i = 1; i < n; ++i) {
      const float x = lam[i];
      int j = i - 1;
      while (j >= 0 && lam[j] < x) {
        lam[j + 1] = lam[j];
        --j;
      }
      lam[j + 1] = x;
    }
    const float s1 = sqrtf(lam[0]);
    for (int i = 0; i < 64; ++i) {
      const float si = (i < n) ? sqrtf(lam[i]) : 0.f;
      f[i] = (s1 > 0.f && si > s1 * 1e-16f) ? log10f(si / s1) : -16.f;
    }
    const double nm = sqrt(fmax(*norm2, 0.0));
    f[64] = (nm > 0.0) ? (float)log10(fmax(tol, 1e-300) / nm) : 16.f;
    f[65] = (float)(log2((double)c) / 10.0);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_mlp_round_input(const float* X, int64_t n, __nv_bfloat16* out, cudaStream_t s) {
  ProfScope prof(K_MLP, s);
  round_input_kernel<<<grid1(n), MT, 0, s>>>(X, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_linear(const __nv_bfloat16* in, int64_t B, int nin, const __nv_bfloat16* W, const float* bias,
                              int nout, float* pre, __nv_bfloat16* act, float* out, cudaStream_t s) {
  ProfScope prof(K_MLP, s, 2.0 * (double)B * nin * nout, 2.0 * (double)B * (nin + nout));
  linear_fwd_kernel<<<grid1(B * nout), MT, 0, s>>>(in, B, nin, W, bias, nout, pre, act, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss(const float* o, const float* T, int64_t B, float* dO, double* loss, cudaStream_t s) {
  ProfScope prof(K_MLP, s);
  loss_kernel<<<grid1(B), MT, 0, s>>>(o, T, B, dO, loss);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_outer(const float* A, int64_t B, int R, const __nv_bfloat16* Bm, int C, float* G, float* gb,
                             cudaStream_t s) {
  ProfScope prof(K_MLP, s, 2.0 * (double)B * R * C, 0.0);
  outer_reduce_kernel<<<grid1((int64_t)R * C), MT, 0, s>>>(A, B, R, Bm, C, G, gb);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_backprop(const float* dA, int64_t B, int J, const __nv_bfloat16* W, int I, const float* pre,
                                float* D, cudaStream_t s) {
  ProfScope prof(K_MLP, s, 2.0 * (double)B * J * I, 0.0);
  backprop_kernel<<<grid1(B * I), MT, 0, s>>>(dA, B, J, W, I, pre, D);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, float c1, float c2,
                            cudaStream_t s) {
  ProfScope prof(K_MLP, s);
  adam_kernel<<<grid1(n), MT, 0, s>>>(w, m, v, g, n, lr, c1, c2, 0.9f, 0.999f, 1e-8f);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_to_bf16(const float* w, int64_t n, __nv_bfloat16* out, cudaStream_t s) {
  ProfScope prof(K_MLP, s);
  to_bf16_kernel<<<grid1(n), MT, 0, s>>>(w, n, out);
  note_launch();
  return cudaGetLastError();
}

size_t sketch_workspace_bytes(int64_t c, int k) {
  return sizeof(float) * ((size_t)c * k * 2 + (size_t)k * k) + 256;
}

cudaError_t launch_sketch_features(const double* G, int64_t c, int k, double tol, const double* norm2, uint64_t seed,
                                   void* work, float* feat, cudaStream_t s) {
  if (c <= 0 || k <= 0 || k > 128) return cudaErrorInvalidValue;
  float* Om = static_cast<float*>(work);
  float* T = Om + (size_t)c * k;
  float* S = T + (size_t)c * k;
  ProfScope prof(K_MLP, s, 2.0 * (double)c * c * k + 2.0 * (double)k * k * c, 8.0 * (double)c * c);
  gauss_sketch_kernel<<<grid1(c * k), MT, 0, s>>>(Om, c, k, seed);
  sketch_left_kernel<<<grid1((int64_t)k * c), MT, 0, s>>>(G, c, Om, k, T);
  sketch_right_kernel<<<grid1((int64_t)k * k), MT, 0, s>>>(T, c, Om, k, S);
  // k x k sketch Gram; when c < k its eigenvalues beyond the c-th are zero
  const size_t sm = sizeof(float) * ((size_t)k * k + k);
  cudaError_t e = allow_max_smem(reinterpret_cast<const void*>(jacobi_features_kernel));
  if (e != cudaSuccess) return e;
  jacobi_features_kernel<<<1, 256, sm, s>>>(S, k, tol, norm2, c, feat);
  note_launch();
  return cudaGetLastError();
}

}  // namespace bht

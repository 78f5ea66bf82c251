// internal.cuh — declarations shared by the library's translation units.
// Not part of the C ABI (include/bht.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bht {

// Launch counter (kernels launched by the library on the calling thread).
void note_launch(int n = 1);

// Kernel classes timed by the optional per-launch CUDA-event profiler.
enum KernelClass {
  K_GRAM_F64 = 0,
  K_TTM_F64 = 1,
  K_EIG_SMALL = 2,
  K_EIG_COOP = 3,
  K_GEMM_F64 = 4,
  K_NORM = 5,
  K_COPY = 6,
  K_TTM_TC = 7,
  K_GRAM_F32 = 8,
  K_OTHER = 9,
  K_NUM_CLASSES = 10
};
const char* kernel_class_name(int cls);

// Records a CUDA event pair around one launch on `s` when the class is enabled.
// `flops` and `bytes` are the algorithmic work of the launch (what the math
// requires, not what the kernel happens to do), summed per class.
struct ProfScope {
  ProfScope(int cls, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
  ~ProfScope();
  int cls_;
  cudaStream_t s_;
  bool on_;
  cudaEvent_t e0_ = nullptr;
};

// Status word written by kernels that can fail on the device (bounded waits,
// non-finite data). 0 = fine; otherwise a bht_status code.
struct DevStatus {
  int* word = nullptr;  // device int
};

// ---------------------------------------------------------------------------
// FP64 / SIMT dense kernels (dense.cu)
//
// A tensor view [A][I][B] (row-major, contiguous) stands for the mode
// unfolding of a layer intermediate: rows I are the node's index, columns the
// (a, b) pairs, a = items x preceding node indices, b = following node indices.
// ---------------------------------------------------------------------------

// G[i][j] += sum_{a,b} X[a][i][b] X[a][j][b]  (G is I x I FP64, zeroed by the caller)
template <typename T>
cudaError_t launch_gram_f64(const T* X, double* G, int64_t A, int64_t I, int64_t B,
                            cudaStream_t s);

// out[a][s][b] = sum_t M(s, t) X[a][t][b], M(s, t) = M[s * ms + t * mt], s < S, t < T.
template <typename Tin, typename Tout>
cudaError_t launch_ttm_f64(const Tin* X, Tout* out, const double* M, int64_t ms, int64_t mt,
                           int64_t A, int64_t T, int64_t B, int64_t S, cudaStream_t s);

// *acc += sum_i x_i^2 (acc is a device double, not zeroed here)
template <typename T>
cudaError_t launch_sqnorm(const T* x, int64_t n, double* acc, cudaStream_t s);

// *acc += trace of the n x n matrix G
cudaError_t launch_trace(const double* G, int64_t n, double* acc, cudaStream_t s);

// C(m, n) = alpha * sum_k A(m, k) B(k, n) + beta * C(m, n), FP64, every operand
// given by (row stride, column stride); M, N, K small to moderate.
cudaError_t launch_gemm_f64(int64_t M, int64_t N, int64_t K, double alpha,
                            const double* A, int64_t a_rs, int64_t a_cs,
                            const double* B, int64_t b_rs, int64_t b_cs, double beta,
                            double* C, int64_t c_rs, int64_t c_cs, cudaStream_t s);

// out[a][b][c] (dims A2 x B2 x C2) = in[a][b][c] if a < A1, b < B1, c < C1 else 0.
template <typename Tin, typename Tout>
cudaError_t launch_copy_pad3(const Tin* in, int64_t A1, int64_t B1, int64_t C1,
                             Tout* out, int64_t A2, int64_t B2, int64_t C2, cudaStream_t s);

// out[i][j] = in[i * ld_in + j] for i < rows, j < cols (column block copy, FP64)
cudaError_t launch_copy_cols(const double* in, int64_t ld_in, int64_t rows, int64_t cols,
                             double* out, int64_t ld_out, cudaStream_t s);

// out[i] = (Tout) in[i]
template <typename Tin, typename Tout>
cudaError_t launch_cast(const Tin* in, Tout* out, int64_t n, cudaStream_t s);

// Symmetric orthonormalisation helper: W (k x k) <- W * diag(1/sqrt(max(lam, tiny)))
cudaError_t launch_scale_cols_invsqrt(double* W, int64_t k, const double* lam, cudaStream_t s);

// A (n x n) <- identity
cudaError_t launch_fill_identity(double* A, int64_t n, cudaStream_t s);

// Flag non-finite entries of x into *flag (set to 1).
template <typename T>
cudaError_t launch_check_finite(const T* x, int64_t n, int* flag, cudaStream_t s);

// ---------------------------------------------------------------------------
// FP64 symmetric eigensolvers (eig.cu)
// ---------------------------------------------------------------------------

// Full eigendecomposition of a symmetric n x n FP64 matrix G (overwritten).
// lam[0..n-1] receive the eigenvalues in descending order; V ([n][n] row-major)
// receives the matching eigenvectors as columns. work must hold
// eig_workspace_bytes(n) bytes. status: device int, set to a bht_status code
// on a failed bounded wait.
size_t eig_workspace_bytes(int64_t n);
cudaError_t launch_eig_sym(double* G, int64_t n, double* lam, double* V, void* work,
                           int* status, cudaStream_t s);

}  // namespace bht

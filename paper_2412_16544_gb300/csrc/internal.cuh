// internal.cuh — declarations shared by the library's translation units.
// Not part of the C ABI (include/bht.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace bht {

// Launch counter (kernels launched by the library on the calling thread).
void note_launch(int n = 1);

// Message returned by bht_last_error() on the calling thread.
void set_last_error(const char* msg);

// Kernel classes timed by the optional per-launch CUDA-event profiler.
enum KernelClass {
  K_GRAM_F64 = 0,
  K_TTM_F64 = 1,
  K_EIG_TRIDIAG = 2,
  K_EIG_BISECT = 3,
  K_GEMM_F64 = 4,
  K_NORM = 5,
  K_COPY = 6,
  K_TTM_TC = 7,
  K_GRAM_F32 = 8,
  K_EIG_INVIT = 9,
  K_EIG_BACK = 10,
  K_TTM_F32 = 11,
  K_HOUSE = 12,
  K_MLP = 13,
  K_PREP = 14,
  K_OTHER = 15,
  K_PAIR_PROJ = 16,  // two-mode projections of small leaves (pair.cu)
  K_PAIR_GRAM = 17,  // two-mode Gram passes (pair.cu)
  K_SPD = 18,        // full-rank certificates by Cholesky factorisation (chol.cu)
  K_TRI_PROJ = 19,   // three-mode projections (tri.cu)
  K_RITZ = 20,       // small eigenproblems by FP32 Jacobi and FP64 Ritz values (ritz.cu)
  K_NUM_CLASSES = 21
};
const char* kernel_class_name(int cls);

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum, once per kernel and
// device, under a lock. The cap belongs to the function and is shared by every host thread; a value
// set per launch by one thread could be lowered by another between its occupancy query and its
// launch, so it is only ever raised. Call before every launch with dynamic shared memory (dynamic
// plus static must fit the cap, and the default cap is 48 KB).
cudaError_t allow_max_smem(const void* func);

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

// Same Gram with FP32 products, partial sums promoted to FP64 every 16 columns.
cudaError_t launch_gram_f32(const float* X, double* G, int64_t A, int64_t I, int64_t B, cudaStream_t s);

// FP32 SIMT mode product with an FP32 matrix M(s, t) = M[s * ms + t * mt]; with
// B == 1 the new axis is written in front of the last R2 rows:
// out[(o * S + s) * R2 + i] for a = o * R2 + i (R2 = 1: in place).
template <typename Tin>
cudaError_t launch_ttm_f32(const Tin* X, float* out, const float* M, int64_t ms, int64_t mt, int64_t A, int64_t T,
                           int64_t B, int64_t S, int64_t R2, cudaStream_t s);

// x <- H_0 H_1 ... H_{K-1} x for nvec vectors of length L (wy.cu), H_k = I - tau_k v_k v_k^T with v_k
// zero above row k + off (off 0 or 1), 1 at that row, and its entry i stored at
// V[k * ldv + i - rel * (k + off)] (rel 0: absolute rows; rel 1: from position 0). Vector c is
// X[i * xrs + c] (X null: the unit vector e_{unit0 + c}) and is written to out[i * ors + c]; X and out
// may be the same matrix. K <= L <= 4096. work: wy_workspace_bytes(K) bytes (the block factors).
size_t wy_workspace_bytes(int64_t K);
cudaError_t launch_wy_apply(const double* V, int64_t ldv, int off, int rel, const double* tau, int64_t K, int64_t L,
                            const double* X, int64_t xrs, int64_t unit0, int64_t nvec, double* out, int64_t ors,
                            void* work, cudaStream_t s);

// Householder complement: out (a x (c - k)) = Q (a x c) times the last c - k columns of the
// orthogonal factor of the QR factorisation of Z (c x k, orthonormal columns). work: at least
// house_workspace_bytes(c, k, #SM) bytes; status: device word of the bounded grid barrier.
size_t house_workspace_bytes(int64_t c, int64_t k, int nsm);
cudaError_t launch_house_complement(const double* Q, int64_t a, int64_t c, const double* Z, int64_t k, double* out,
                                    void* work, int* status, cudaStream_t s);

// The same with S computed output columns of which the first S_store are stored (the new axis has
// S_store entries); the squares of the others are added to *resid (nullable, FP64).
template <typename Tin>
cudaError_t launch_ttm_f32_resid(const Tin* X, float* out, const float* M, int64_t ms, int64_t mt, int64_t A,
                                 int64_t T, int64_t B, int64_t S, int64_t S_store, int64_t R2, double* resid,
                                 cudaStream_t s);

// ---------------------------------------------------------------------------
// Rank / expansion predictor (mlp.cu): bf16 weights and activations, FP32 accumulation.
// ---------------------------------------------------------------------------
cudaError_t launch_mlp_round_input(const float* X, int64_t n, __nv_bfloat16* out, cudaStream_t s);
cudaError_t launch_mlp_linear(const __nv_bfloat16* in, int64_t B, int nin, const __nv_bfloat16* W, const float* bias,
                              int nout, float* pre, __nv_bfloat16* act, float* out, cudaStream_t s);
cudaError_t launch_mlp_loss(const float* o, const float* T, int64_t B, float* dO, double* loss, cudaStream_t s);
cudaError_t launch_mlp_outer(const float* A, int64_t B, int R, const __nv_bfloat16* Bm, int C, float* G, float* gb,
                             cudaStream_t s);
cudaError_t launch_mlp_backprop(const float* dA, int64_t B, int J, const __nv_bfloat16* W, int I, const float* pre,
                                float* D, cudaStream_t s);
cudaError_t launch_mlp_adam(float* w, float* m, float* v, const float* g, int64_t n, float lr, float c1, float c2,
                            cudaStream_t s);
cudaError_t launch_mlp_to_bf16(const float* w, int64_t n, __nv_bfloat16* out, cudaStream_t s);
// 66 features of the node whose Gram matrix is G (c x c, FP64): log10 of the sketched singular values
// relative to the largest (64), log10(tol / sqrt(*norm2)) with norm2 on the device, log2(c) / 10.
// work: sketch_workspace_bytes(c, k).
size_t sketch_workspace_bytes(int64_t c, int k);
cudaError_t launch_sketch_features(const double* G, int64_t c, int k, double tol, const double* norm2, uint64_t seed,
                                   void* work, float* feat, cudaStream_t s);

// out[s * T + t] = (float) U[s * ms + t * mt]
cudaError_t launch_cast_matrix(const double* U, int64_t ms, int64_t mt, int64_t S, int64_t T, float* out,
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

// W (rows x cols, row-major) <- W * diag(1/sqrt(max(lam, tiny)))
cudaError_t launch_scale_cols_invsqrt(double* W, int64_t rows, int64_t cols, const double* lam, cudaStream_t s);
// Data preparation (prep.cu). Per group g of `size` consecutive elements: params[2g] = shift,
// params[2g + 1] = scale (device), kind 1 max-abs, 2 unit vector, 3 z-score; then y <- (y - shift) / scale.
cudaError_t launch_normalize(void* Y, int dtype, int64_t groups, int64_t size, int kind, double* params,
                             cudaStream_t s);
// y <- y * scale + shift per group.
cudaError_t launch_denormalize(void* Y, int dtype, int64_t groups, int64_t size, const double* params,
                               cudaStream_t s);
// out item n = permutation of item n of Y: out[n][i_{perm[0]}]..[i_{perm[d-1]}] = Y[n][i_0]..[i_{d-1}].
cudaError_t launch_permute_items(const void* Y, int dtype, int64_t N, int d, const int64_t* dims, const int* perm,
                                 void* out, cudaStream_t s);
// err2[n] += ||X_n - Xh_n||^2, nrm2[n] += ||X_n||^2 over items of `item` elements (Xh FP64).
cudaError_t launch_item_errors(const void* X, int dtype, const double* Xh, int64_t N, int64_t item, double* err2,
                               double* nrm2, cudaStream_t s);

// out[a][b][t] = in[a][t][b] (t < T), 0 for T <= t < Tp: the middle axis of fp32 [A][T][B] moved innermost
// and zero padded to Tp.
cudaError_t launch_transpose_pad(const float* in, float* out, int64_t A, int64_t T, int64_t B, int64_t Tp,
                                 cudaStream_t s);
// out = in^T for a row-major [rows][cols] matrix of 4- or 8-byte elements (rows <= 2,097,120).
cudaError_t launch_transpose2d(const void* in, void* out, int64_t rows, int64_t cols, int elem_bytes,
                               cudaStream_t s);

// X[e] <- uniform in [-1, 1) from a counter-based hash of (seed, e); deterministic
cudaError_t launch_fill_uniform(double* X, int64_t n, uint64_t seed, cudaStream_t s);

// Q[j * ldq + col0 + idx(j)] = 1 for the coordinates j = i * rb + k of a merged index grown from
// ra0 x rb0 to ra x rb that are new (i >= ra0 or k >= rb0), idx numbering them in C order.
cudaError_t launch_unit_cols(double* Q, int64_t ldq, int64_t col0, int64_t ra0, int64_t rb0, int64_t ra, int64_t rb,
                             cudaStream_t s);

// A (n x n) <- identity
cudaError_t launch_fill_identity(double* A, int64_t n, cudaStream_t s);

// Flag non-finite entries of x into *flag (set to 1).
template <typename T>
cudaError_t launch_check_finite(const T* x, int64_t n, int* flag, cudaStream_t s);

// ---------------------------------------------------------------------------
// FP64 symmetric eigensolvers (eig.cu)
// ---------------------------------------------------------------------------

// Two-stage eigensolver of a symmetric n x n FP64 matrix G (n <= 4096).
// Stage 1 overwrites G, keeps the tridiagonal form and its reflectors in
// `work` (eig_workspace_bytes(n)) and writes every eigenvalue, descending,
// to lam. Stage 2 (same `work`, after stage 1) writes the eigenvectors of the
// r largest eigenvalues as the columns of U ([n][r] row-major), using
// `scratch` (eig_vectors_scratch_bytes(n, r)). status: device int, set to a
// bht_status code when a bounded wait gives up.
size_t eig_workspace_bytes(int64_t n);
size_t eig_vectors_scratch_bytes(int64_t n, int64_t r);
cudaError_t launch_eig_values(double* G, int64_t n, double* lam, void* work, int* status, cudaStream_t s);
// Stage 1 split in two: the tridiagonalisation (G overwritten), then the eigenvalues with
// descending indices [j0, j1) only (lam[j] = j-th largest). The diagonal of T (device, n doubles)
// gives trace(G) for tail sums without the small eigenvalues.
cudaError_t launch_eig_tridiag(double* G, int64_t n, void* work, int* status, cudaStream_t s);
cudaError_t launch_eig_bisect(int64_t n, void* work, double* lam, int64_t j0, int64_t j1, cudaStream_t s);
const double* eig_tridiag_diagonal(void* work, int64_t n);
cudaError_t launch_eig_vectors(int64_t n, int64_t r, const double* lam, double* U, void* work, void* scratch,
                               cudaStream_t s);

// ---------------------------------------------------------------------------
// tcgen05 tensor-core mode product over the innermost axis (tc.cu)
//   out[(o * S + s) * R2 + i] = sum_k X[o * R2 + i][k] U[k][s]
// X fp32 [rows][K] (K % 4 == 0, 16-byte aligned); W prepared by
// launch_prep_tc_weights from the FP64 basis (nb = 1: TF32 of U^T;
// nb = 2: TF32 of U^T plus its TF32 remainder). norm_in / norm_out (nullable,
// device doubles) accumulate ||X||^2 and ||out||^2 in FP64.
// ---------------------------------------------------------------------------
bool ttm_tc_supported(int64_t K, int64_t S, int nb);
size_t ttm_tc_weights_bytes(int64_t K, int64_t S);
cudaError_t launch_prep_tc_weights(const double* U, int64_t K, int64_t S, int64_t ldu, bool transpose, float* W,
                                   int nb, cudaStream_t s);
cudaError_t launch_ttm_tc(const float* X, int64_t rows, int64_t K, const float* W, int64_t S, int nb, float* out,
                          int64_t R2, double* norm_in, double* norm_out, int* status, cudaStream_t s);
// Weights of the concatenated matrix M = [U | U2] (S1 + S2 output columns; U [K][S1] with row stride
// ldu when transpose, U2 likewise).
cudaError_t launch_prep_tc_weights2(const double* U, int64_t S1, int64_t ldu, const double* U2, int64_t S2,
                                    int64_t ldu2, int64_t K, bool transpose, float* W, int nb, cudaStream_t s,
                                    int64_t k_valid = -1);
// S computed output columns of which the first S_store are stored (the output's new axis has S_store
// entries); the squares of the other S - S_store columns are added to *resid (nullable, FP64).
cudaError_t launch_ttm_tc_resid(const float* X, int64_t rows, int64_t K, const float* W, int64_t S, int64_t S_store,
                                int nb, float* out, int64_t R2, double* norm_in, double* norm_out, double* resid,
                                int* status, cudaStream_t s);

// ---------------------------------------------------------------------------
// Two-mode passes over X[A][na][nb][B] (pair.cu): TMA-staged tiles, FP32 SIMT or tensor cores, one read
// of X (the tensor-core Gram reads each tile a second time, from L2).
// ---------------------------------------------------------------------------
bool pair_gram_supported(int64_t A, int64_t na, int64_t nb, int64_t B);
bool pair_project_supported(int64_t A, int64_t na, int64_t nb, int64_t B, int64_t ra, int64_t rb);
// G_a (na x na) and G_b (nb x nb) += the Gram matrices of the two mode unfoldings (zeroed by the caller).
// tensor_cores: the split-TF32 tcgen05 pass where the shape has one (na = nb = 24), else FP32 SIMT.
cudaError_t launch_pair_gram(const float* X, int64_t A, int na, int nb, int64_t B, double* Ga, double* Gb,
                             int* status, cudaStream_t s, bool tensor_cores);
// out[A][ra][rb][B] = X x_a Ua^T x_b Ub^T (Ua [na][ra] with leading dimension lda, Ub likewise);
// norm_in += ||X||^2, norm_out += ||out||^2, resid += their difference (each nullable).
cudaError_t launch_pair_project(const float* X, int64_t A, int na, int nb, int64_t B, const double* Ua, int ra,
                                int lda, const double* Ub, int rb, int ldb, float* out, double* norm_in,
                                double* norm_out, double* resid, int* status, cudaStream_t s);

// A (n x n) += alpha I
// out[A][r1][r2][r3] (fp32) = X x_1 U1^T x_2 U2^T x_3 U3^T for X fp32 [A][n1][n2][n3] (16-byte aligned,
// slabs contiguous) and FP64 bases U_m [n_m][r_m] (row stride ld_m); norm_in, norm_out, resid (nullable
// FP64 device accumulators) receive ||X||^2, ||out||^2 and their difference added (tri.cu).
bool tri_project_supported(int64_t A, int64_t n1, int64_t n2, int64_t n3, int64_t r1, int64_t r2, int64_t r3);
cudaError_t launch_tri_project(const float* X, int64_t A, int n1, int n2, int n3, const double* U1, int r1, int ld1,
                               const double* U2, int r2, int ld2, const double* U3, int r3, int ld3, float* out,
                               double* norm_in, double* norm_out, double* resid, int* status, cudaStream_t s);

// Eigenpairs of the symmetric n x n FP64 matrix G (device, n <= 32) for a mixed-precision truncation:
// lam[n] the Ritz values of FP32 Jacobi vectors made orthonormal in FP64, in decreasing order, and
// V[n][n] (row-major) those vectors in the same order (ritz.cu).
cudaError_t launch_small_ritz(const double* G, int64_t n, double* lam, double* V, cudaStream_t s);

// Certificate that every eigenvalue of the symmetric n x n FP64 matrix G (device, row-major; lower
// triangle read) exceeds tau >= 0: *verdict (device int) = 1 when the Cholesky factorisation of
// G - (tau + 2 (n + 4) 2^-53 trace(G)) I completes in FP64, 0 otherwise (chol.cu). n <= 4096; work holds
// spd_test_workspace_bytes(n); status: device word of the bounded grid barrier.
size_t spd_test_workspace_bytes(int64_t n);
cudaError_t launch_spd_test(const double* G, int64_t n, double tau, void* work, int* verdict, int* status,
                            cudaStream_t s);
cudaError_t launch_add_diag(double* A, int64_t n, double alpha, cudaStream_t s);

}  // namespace bht

/*
 * bht.h — C ABI of the GB300 batch hierarchical Tucker library (libbht.so).
 *
 * The library compresses a stream of tensor batches into the batch
 * hierarchical Tucker (batch-HT) format of arXiv 2412.16544:
 *   - bht_l2r        : one-shot leaves-to-root decomposition of a first batch
 *                      (Algorithm 1, "BHT-l2r"; Problem 1, Section 1);
 *   - htrise_update  : incremental update with a new batch, never storing or
 *                      rebuilding the accumulation (Algorithm 2, "HT-RISE";
 *                      Problem 2, Section 1);
 *   - ht_reconstruct : root-to-leaves decoding of stored items
 *                      (eq. htucker_reconstruction, Section 2.3);
 *   - ht_encode      : latent representation of unseen items on the current
 *                      cores (Step 1 of Algorithm 2, used for the relative
 *                      test error of eq. generalization_performance);
 *   - ht_decode, ht_relative_test_error : latent items back to tensors, and
 *                      the mean per-item relative error of unseen items;
 *   - ht_l2r         : the plain hierarchical Tucker baseline (the batch as a
 *                      leaf, leaves-to-root of Section 2.3.1);
 *   - bht_normalize, bht_denormalize, bht_permute_items : batch preparation
 *                      (per-group normalisation, item axis orders);
 *   - bht_mlp_*, bht_sketch_features : the rank / expansion predictor;
 *   - bht_synth_chebyshev : a device generator of the smooth sensor-grid
 *                      stream used to measure long streams (input synthesis,
 *                      no counterpart in the paper).
 *
 * Conventions shared by every call
 *   - Every function returns bht_status; BHT_OK (0) on success. Nothing is
 *     thrown across the ABI. bht_last_error() returns a thread-local message
 *     describing the last failure of the calling thread.
 *   - Batches are item-major, C-order: element (m, i_1, ..., i_d) of an
 *     N-item batch with modes n_1..n_d sits at offset
 *     ((m * n_1 + i_1) * n_2 + i_2) ... * n_d + i_d. The paper keeps the batch
 *     last; its Section 3.1 footnote states the batch position does not matter.
 *   - Data pointers may be device pointers or host pointers (pinned or
 *     pageable); the library detects which (cudaPointerGetAttributes) and
 *     copies host data through its own device staging buffer on `stream`.
 *     The caller keeps ownership of every pointer it passes and must keep
 *     it valid until the call returns (host data) or until `stream` has
 *     passed the call (device data).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that decide ranks synchronise `stream` before they return.
 *   - The dimension tree is the balanced binary tree over modes 1..d whose
 *     first child of a node with m modes takes ceil(m/2) of them (Fig. 2,
 *     Section 2.3); the batch is not a tree node, it rides on the root
 *     (Section 3.1). Node order everywhere is breadth-first, left to right:
 *     node 0 is the root, nodes 1 and 2 are its successors, ...
 *   - Cores (Section 2.3): a leaf core is U in R^{n x r}, row-major [n][r];
 *     a transfer core is G in R^{r_l x r_r x r}, C-order [r_l][r_r][r]
 *     (the merged row index is i_l * r_r + i_r); the root is stored item-major
 *     [N_total][r_11][r_12].
 *   - Errors: on any error inside htrise_update the state is left exactly as
 *     it was before the call (updates are built in fresh buffers and
 *     committed only at the end).
 *   - Environment: BHT_AUTOTUNE=1 lets the library time the launch shapes of
 *     its tridiagonalisation per matrix-size bucket and keep the fastest for
 *     the process (off by default).
 */
#ifndef BHT_H_
#define BHT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BHT_OK = 0,
  BHT_EINVAL = 1,        /* invalid argument (null pointer, bad size, d < 2, eps <= 0) */
  BHT_ENOMEM = 2,        /* device or host allocation failed */
  BHT_ECAPACITY = 3,     /* a size exceeds a documented maximum */
  BHT_ECUDA = 4,         /* a CUDA runtime call failed; see bht_last_error() */
  BHT_ENUMERIC = 5,      /* non-finite values in the input or in an intermediate */
  BHT_ETIMEOUT = 6,      /* a bounded device-side wait gave up; results are invalid */
  BHT_EUNSUPPORTED = 7   /* a valid request this build does not implement */
} bht_status;

/* Element type of a batch or of an output buffer. */
typedef enum { BHT_F32 = 0, BHT_F64 = 1 } bht_dtype;

/* Arithmetic of the path.
 *   BHT_PREC_FP64 : every contraction, Gram matrix, eigensolve and norm in FP64
 *                   (the plain GPU form of the method).
 *   BHT_PREC_MIXED: mode products of an innermost axis on tcgen05 tensor
 *                   cores (split TF32: three TF32 products, FP32
 *                   accumulation), other mode products in FP32, Gram matrices
 *                   with FP32 products summed in FP64 (FP64 Grams when
 *                   eps_rel < 1e-3); node eigensolves, re-orthogonalisation,
 *                   norms and the skip test stay in FP64. */
typedef enum { BHT_PREC_FP64 = 0, BHT_PREC_MIXED = 1 } bht_precision;

/* Node-wise error budget.
 *   BHT_BUDGET_UNIFORM : eps_nw = eps_abs / sqrt(2d - 2) at every truncation (Algorithms 1, 2).
 *   BHT_BUDGET_ADAPTIVE: after each layer the error actually spent, eps_l^2 = ||Y||^2 - ||C_l||^2, is
 *                        measured and eps_nw = sqrt(eps_abs^2 - eps_l^2) / sqrt(truncations left)
 *                        (App. C). The bound ||Y - Y~|| <= eps_abs holds for both. */
typedef enum { BHT_BUDGET_UNIFORM = 0, BHT_BUDGET_ADAPTIVE = 1 } bht_budget;

typedef struct bht_tree bht_tree;
typedef struct bht_state bht_state;
/* Rank / expansion predictor (no counterpart in the paper): a three-layer perceptron with bf16
 * weights and activations, see bht_mlp_create. */
typedef struct bht_mlp bht_mlp;

/* Options of bht_l2r / htrise_update; NULL means all defaults (FP64, no predictor). */
typedef struct {
  int32_t precision;      /* bht_precision */
  int32_t budget;         /* bht_budget, or -1: bht_l2r uniform, htrise_update the state's (the budget
                             given to bht_l2r) */
  /* htrise_update only. With a predictor, every node whose residual Gram matrix is formed gets its
   * 66 sketch features and a prediction; a node predicted not to expand skips its residual
   * eigensolve when the exact residual energy trace(R R^T) <= eps_nw^2 confirms that the truncation
   * of eq. svd_on_residual keeps nothing (the exact check), and is truncated as usual otherwise (the
   * fallback). The result is the same as without the predictor. */
  const bht_mlp* predictor;
  /* Optional host outputs, one row per tree node (node ids as bht_get_ranks), written for every
   * node whose residual was formed and left untouched for the others: node_features [nodes][66]
   * (fp32) and node_labels [nodes][2] (int64: residual rank r_R kept, residual dimension). They
   * are the training pairs the method generates for the predictor. */
  float* node_features;
  int64_t* node_labels;
} bht_opts;

/* Outcome of one htrise_update call. */
typedef struct {
  int32_t skipped;        /* 1: projection error <= eps_des, only the root grew (Algorithm 2) */
  int32_t batch_reads;    /* kernels of this call that read the whole new batch (passes over Y) */
  double eps_proj;        /* projection error of eq. relative_error_threshold (FP64: sqrt(max(||Y||^2 -
                             ||C_1||^2, 0)); mixed: square root of the energy removed on the nodes'
                             complements) */
  double eps_des;         /* eps_rel * ||Y||_F of the new batch */
  double norm_y;          /* ||Y||_F of the new batch */
  int64_t n_items_total;  /* items in the accumulation after the call */
  int32_t pred_nodes;     /* nodes the predictor saw */
  int32_t pred_skipped;   /* of those, residual eigensolves skipped (prediction confirmed by the exact check) */
  int32_t pred_fallback;  /* predicted "no expansion" but the exact check found residual energy above eps_nw^2 */
  int32_t pred_missed;    /* predicted "expands" but the truncation kept nothing */
} bht_update_info;

/* Balanced binary dimension tree over d >= 2 modes of sizes dims[0..d-1]
 * (Section 2.3, Fig. 2). `out` receives a host object owned by the caller,
 * released with bht_tree_destroy. d <= 16 and every dims[i] in [1, 4096]. */
bht_status bht_tree_create_balanced(int32_t d, const int64_t* dims, bht_tree** out);
bht_status bht_tree_destroy(bht_tree* tree);
/* Depth p and number of nodes 2d-1 of a tree. */
bht_status bht_tree_info(const bht_tree* tree, int32_t* depth, int32_t* num_nodes);

/* BHT-l2r (Algorithm 1): compress a first batch Y of N items into a new state.
 *   Y      : [N][n_1]..[n_d] item-major, element type `dtype`, device or host.
 *   eps_rel: relative tolerance; the result satisfies ||Y - Y~|| <= eps_rel ||Y||
 *            (Corollary bht_leaves_to_root) up to the arithmetic of `opts`.
 *   opts   : may be NULL (= BHT_PREC_FP64).
 *   out    : receives a state owned by the caller (bht_state_destroy). The
 *            state keeps its own copy of the tree. */
bht_status bht_l2r(const bht_tree* tree, const void* Y, int32_t dtype, int64_t N,
                   double eps_rel, const bht_opts* opts, void* stream, bht_state** out);

/* Plain hierarchical Tucker baseline (the leaves-to-root algorithm of Sec. 2.3.1, one-shot): the N
 * items are one (d+1)-mode tensor with the batch as the LAST leaf of the balanced tree over
 * (n_1, .., n_d, N) (Fig. htucker_as_node), truncated with eps_nw = eps_rel ||Y|| / sqrt(2(d+1) - 3)
 * (Theorem ht_nodewise_error).
 *   dims   : the d item mode sizes, each in [1, 4096]; 2 <= d <= 15.
 *   Y      : [N][n_1]..[n_d] item-major, element type `dtype`, device or host; 1 <= N <= 4096.
 *   opts   : precision as for bht_l2r; the budget must be uniform (BHT_EINVAL otherwise).
 *   out    : a state of one tensor: bht_get_dims reports (n_1, .., n_d, N), bht_get_ranks[0] = 1, the
 *            root is the r_11 x r_12 matrix of the last truncation, and ht_reconstruct(state, 0, 1)
 *            writes the tensor with the batch last, [n_1]..[n_d][N]. htrise_update and ht_encode
 *            return BHT_EINVAL on it. */
bht_status ht_l2r(int32_t d, const int64_t* dims, const void* Y, int32_t dtype, int64_t N, double eps_rel,
                  const bht_opts* opts, void* stream, bht_state** out);

/* HT-RISE (Algorithm 2): update `state` with a new batch of N items.
 *   Projects Y onto the current cores; if the projection error is <= eps_rel ||Y||
 *   only the root grows, otherwise residuals are truncated node by node, the
 *   bases expanded and re-orthogonalised, parents zero-padded and the batch
 *   re-projected. `info` may be NULL. */
bht_status htrise_update(bht_state* state, const void* Y, int32_t dtype, int64_t N,
                         double eps_rel, const bht_opts* opts, void* stream,
                         bht_update_info* info);

/* HT-RISE (Algorithm 2) over a stream of `count` batches of N items each, in order: the same result
 * as `count` calls of htrise_update on consecutive batches, with the GPU kept busy between them.
 *   Y      : [count][N][n_1]..[n_d] item-major, element type `dtype`, device or host. Host batches
 *            are copied into two device buffers on a copy stream of the call while the previous
 *            batch computes (pinned host memory lets the copies overlap; pageable memory works but
 *            serialises them).
 *   infos  : NULL or [count] outcomes, one per batch, as htrise_update reports them.
 *   done   : NULL or the number of batches committed when the call returns (count on success).
 *   Step 1 of batch k + 1 (its projection onto the current cores) is enqueued before the skip test
 * of batch k is read back: when batch k is skipped the cores do not change and that projection is the
 * one Algorithm 2 makes; when batch k expands them, it is dropped and made again on the new cores.
 * On an error the state holds every batch before the failing one (*done of them) and none after.
 * opts as for htrise_update; its per-node outputs describe the last batch that expanded the cores.
 * Synchronises `stream` before it returns. */
bht_status htrise_update_stream(bht_state* state, const void* Y, int32_t dtype, int64_t N, int64_t count,
                                double eps_rel, const bht_opts* opts, void* stream, bht_update_info* infos,
                                int64_t* done);

/* Root-to-leaves reconstruction (eq. htucker_reconstruction) of stored items
 * first .. first+count-1 into `out` ([count][n_1]..[n_d], element type `dtype`,
 * device or host). Never modifies the state. */
bht_status ht_reconstruct(const bht_state* state, int64_t first, int64_t count,
                          void* out, int32_t dtype, void* stream);

/* Root-to-leaves expansion of N latent items (FP64 [N][r_11][r_12], host or device, e.g. from
 * ht_encode) into `out` ([N][n_1]..[n_d], element type `dtype`, host or device). With ht_encode this
 * gives the relative test error ||X - decode(encode(X))|| / ||X|| of unseen items. N = 0 does
 * nothing; N < 0 is BHT_EINVAL. Never modifies the state. Synchronises `stream`. */
bht_status ht_decode(const bht_state* state, const double* latent, int64_t N, void* out, int32_t dtype,
                     void* stream);

/* Relative test error of N items X (eq. generalization_performance): each item is encoded (Step 1
 * of Algorithm 2) and decoded (eq. htucker_reconstruction) on the current cores and the per-item
 * relative errors ||X_i - X~_i|| / ||X_i|| are averaged into *rte (host). item_err (host, [N]) may be
 * NULL, else receives the per-item errors; an all-zero item that decodes to zero counts 0.
 * X: [N][n_1]..[n_d], element type `dtype`, host or device; N >= 1. BHT_EINVAL on a plain HT state.
 * Works in chunks of at most 2^27 decoded elements. Synchronises `stream`. */
bht_status ht_relative_test_error(const bht_state* state, const void* X, int32_t dtype, int64_t N, double* rte,
                                  double* item_err, void* stream);

/* Normalisation of snapshots before compression, in place on device memory: Y holds `groups`
 * consecutive groups of `group_size` elements (one group per item, or per item and physical
 * quantity) and every group is normalised on its own, y <- (y - shift) / scale, with
 *   BHT_NORM_MAXABS : shift 0, scale max |y|;
 *   BHT_NORM_UNITVEC: shift 0, scale ||y||_2;
 *   BHT_NORM_ZSCORE : shift mean(y), scale the population standard deviation of y;
 *   BHT_NORM_NONE   : Y unchanged, params (0, 1).
 * A scale that is zero or not finite is replaced by 1. params ([groups][2] FP64 (shift, scale),
 * host or device) receives the parameters for bht_denormalize. Synchronises `stream`. */
typedef enum { BHT_NORM_NONE = 0, BHT_NORM_MAXABS = 1, BHT_NORM_UNITVEC = 2, BHT_NORM_ZSCORE = 3 } bht_norm;
bht_status bht_normalize(void* Y, int32_t dtype, int64_t groups, int64_t group_size, int32_t kind, double* params,
                         void* stream);
/* Inverse of bht_normalize: y <- y * scale + shift per group (params host or device). */
bht_status bht_denormalize(void* Y, int32_t dtype, int64_t groups, int64_t group_size, const double* params,
                           void* stream);

/* Reordering of the item axes (the axis-ordering study of App. D): out[n] is item n of Y with its
 * axes permuted, out axis k = input axis perm[k], so out has the item shape (dims[perm[0]], ..,
 * dims[perm[d-1]]). Y and out: distinct device buffers of N items; 1 <= d <= 16. Synchronises
 * `stream`. */
bht_status bht_permute_items(const void* Y, int32_t dtype, int64_t N, int32_t d, const int64_t* dims,
                             const int32_t* perm, void* out, void* stream);

/* Device generator of the smooth sensor-grid stream (input synthesis; the paper has no counterpart:
 * its cyber-physical experiments read recorded data, which this stands in for). Item j of `count`:
 *     item[i_1..i_d] = sum_{q < terms} prod_{m < d} f_qm(i_m) + noise_std * z_j(e),
 *     f_qm(i) = sum_{k <= degree} coeffs[j][q][m][k] T_k(x_i),  x_i = -1 + 2 i / (n - 1),
 * T_k the Chebyshev polynomials and e the element's C-order index within the item. z is a
 * counter-based standard normal: with b = mix64(seed * 2^32 + first_item + j) and word w_k =
 * mix64(b + (k + 1) * 0x9E3779B97F4A7C15) (SplitMix64's output function mix64; Steele, Lea and
 * Flood, OOPSLA 2014), u1 = (bits 40..63 of w_k + 1/2) / 2^24, u2 = (bits 8..31 + 1/2) / 2^24,
 * z(2k) = sqrt(-2 ln u1) cos(2 pi u2) and z(2k + 1) = sqrt(-2 ln u1) sin(2 pi u2), evaluated in FP32.
 * coeffs: FP64 [count][terms][d][degree + 1], host or device; out: fp32 device
 * [count][n]^d, item-major. 1 <= n <= 64, 2 <= d <= 8, 1 <= terms <= 64, 0 <= degree <= 32,
 * count <= 65535 (0 does nothing); BHT_EINVAL otherwise or when out is not device memory.
 * Asynchronous on `stream` for device coefficients; host coefficients are copied and the call
 * synchronises `stream`. */
bht_status bht_synth_chebyshev(const double* coeffs, int64_t count, int32_t n, int32_t d, int32_t terms,
                               int32_t degree, double noise_std, uint64_t seed, int64_t first_item, float* out,
                               void* stream);

/* Latent representation of N unseen items on the current cores (Step 1 of
 * Algorithm 2), written item-major [N][r_11][r_12] as FP64 into `out`
 * (device or host). N = 0 does nothing; N < 0 is BHT_EINVAL. Never modifies the
 * state. Synchronises `stream`. */
bht_status ht_encode(const bht_state* state, const void* Y, int32_t dtype, int64_t N,
                     double* out, void* stream);

/* One mode product over the innermost axis (eq. ht_leaf_contraction for that
 * axis, Section 2.1 contraction with U^T):
 *     out[(o * S + s) * R2 + i] = sum_k X[(o * R2 + i) * K + k] * U[k * S + s]
 * X: fp32 device [rows][K]; U: FP64 device basis [K][S] (row-major, the
 * layout of a leaf core); out: fp32 device. R2 places the new axis: R2 = 1
 * keeps it innermost, R2 = rows / (item count) moves it in front of the other
 * axes. precision BHT_PREC_MIXED runs the tcgen05 tensor-core kernel (split
 * TF32: x = x_hi + x_lo, U = U_hi + U_lo, three TF32 products, FP32
 * accumulation; K % 4 == 0); BHT_PREC_FP64 the FP64 SIMT kernel (R2 = 1).
 * norms (nullable, device, 2 doubles) receives ||X||^2 and ||out||^2 added
 * in FP64 (mixed only). Synchronises `stream`. */
bht_status bht_mode_product(const float* X, int64_t rows, int64_t K, const double* U, int64_t S,
                            int32_t precision, float* out, int64_t R2, double* norms, void* stream);

/* The two-mode passes of the small leaves (eq. ht_leaf_svd through Gram matrices, and eq.
 * ht_leaf_contraction / Step 1 of Algorithm 2 for two modes at once), exposed for direct tests. X is
 * fp32 device data viewed as [A][na][nb][B] (B contiguous, B % 4 == 0, X 16-byte aligned), read once,
 * tile by tile, through TMA.
 * bht_pair_gram: Ga (na x na) and Gb (nb x nb), FP64 device, receive the Gram matrices of the two
 *   mode unfoldings, G_a = X_(a) X_(a)^T and G_b = X_(b) X_(b)^T. na, nb <= 24. tensor_cores != 0 and
 *   na = nb = 24: tcgen05 MMAs in split TF32 (x = h + l, G = H H^T + L H^T + (L H^T)^T; the missing
 *   L L^T is below 2^-22 of each product), one tile summed in FP32 in tensor memory (96 MMA results
 *   per entry: within 1.2e-5 of the largest entry) and folded into FP64; otherwise, and in BHT-l2r
 *   (where it is 2.7 times faster at 24 x 24), FP32 products with per-lane FP32 partial sums folded
 *   into FP64 (within 2e-6).
 * bht_pair_project: out[A][ra][rb][B] (fp32 device) = X x_a Ua^T x_b Ub^T with Ua [na][ra] and
 *   Ub [nb][rb] FP64 device bases (row-major); norms (nullable, 3 FP64 device values) receives
 *   ||X||^2, ||out||^2 and their difference added in FP64. na, nb <= 32, ra, rb <= 16.
 * Shapes outside these limits give BHT_EUNSUPPORTED. Both synchronise `stream`. */
bht_status bht_pair_gram(const float* X, int64_t A, int64_t na, int64_t nb, int64_t B, double* Ga, double* Gb,
                         int32_t tensor_cores, void* stream);
bht_status bht_pair_project(const float* X, int64_t A, int64_t na, int64_t nb, int64_t B, const double* Ua,
                            int64_t ra, const double* Ub, int64_t rb, float* out, double* norms, void* stream);

/* Three-mode pass (eq. ht_leaf_contraction for three leaves, Step 1 of Algorithm 2): X fp32 device
 * data viewed as [A][n1][n2][n3] (16-byte aligned; the slabs of n1 n2 n3 values contiguous), read once
 * slab by slab. out[A][r1][r2][r3] (fp32 device) = X x_1 U1^T x_2 U2^T x_3 U3^T with U_m [n_m][r_m] FP64
 * device bases (row-major); norms (nullable, 3 FP64 device values) receives ||X||^2, ||out||^2 and their
 * difference added in FP64. Products and sums in FP32. n_m <= 32, r_m <= 8, n2 n3 % 4 == 0 and
 * n1 n2 n3 <= 13824 with the ring of three slabs and the work areas within 220 KB of shared memory;
 * other shapes give BHT_EUNSUPPORTED. Synchronises `stream`. */
bht_status bht_tri_project(const float* X, int64_t A, int64_t n1, int64_t n2, int64_t n3, const double* U1,
                           int64_t r1, const double* U2, int64_t r2, const double* U3, int64_t r3, float* out,
                           double* norms, void* stream);

/* bht_mode_product without any device allocation (the paper has no
 * counterpart: this is an interface for callers that may not allocate device
 * memory during the call, e.g. when another allocator owns the GPU's memory or
 * in a latency-critical loop where cudaMalloc / cudaFree could synchronise).
 * Same operation and arguments as bht_mode_product with precision
 * BHT_PREC_MIXED; X, U, out and norms are the caller's device buffers (a
 * host pointer is BHT_EINVAL, found by a pointer-attribute query that
 * allocates nothing). The
 * scratch (split TF32 weight planes and a status word, 1 MiB + 256 B) is a
 * file-scope device array that every GPU loading the library holds until the
 * process exits; it limits K <= 512 and S <= 256 (BHT_ECAPACITY beyond) and
 * needs K % 4 == 0. The first call on a device looks the array's address up
 * (cudaGetSymbolAddress); make it before any stream capture. All calls share
 * the array and it keeps the last call's contents: calls that overlap on the
 * GPU race on it and must be serialised by the caller. Synchronises `stream`. */
bht_status bht_mode_product_noalloc(const float* X, int64_t rows, int64_t K, const double* U, int64_t S,
                                    float* out, int64_t R2, double* norms, void* stream);

/* Node eigensolver (the error-truncated SVD of eq. ht_leaf_svd taken through
 * the Gram matrix of the unfolding): G is a symmetric FP64 device matrix
 * [n][n] (overwritten); lam receives all n eigenvalues in descending order;
 * U ([n][r] row-major, device) the orthonormal eigenvectors of the r largest
 * ones. n <= 4096. Synchronises `stream`. */
bht_status bht_sym_eig(double* G, int64_t n, double* lam, double* U, int64_t r, void* stream);

/* Eigenpairs for the mixed-precision truncation of a small node (eq. ht_leaf_svd, n <= 32, else
 * BHT_EINVAL): cyclic Jacobi in FP32 on G (n x n symmetric FP64, device, row-major; not written), its
 * vectors made orthonormal in FP64 by two Newton-Schulz steps, and their Ritz values v_i^T G v_i in FP64.
 * lam (device, n) receives the Ritz values in decreasing order and V (device, [n][n] row-major) the
 * vectors as columns in the same order. Keeping the first r columns discards exactly the energy
 * sum_{i>=r} lam_i, the quantity the tail rule bounds; lam differs from the eigenvalues of G by the square
 * of the vectors' FP32-level angles. BHT-l2r uses it in the mixed path for nodes of at most 32 rows.
 * Synchronises `stream`. */
bht_status bht_sym_eig_small(const double* G, int64_t n, double* lam, double* V, void* stream);

/* Full-rank certificate of a truncation (eq. ht_leaf_svd, Algorithm 1): the tail rule keeps all n
 * directions of a node exactly when the smallest eigenvalue of its Gram matrix exceeds the node's
 * budget eps_nw^2. G: n x n symmetric FP64, device, row-major (its lower triangle is read; G itself
 * is not written). *above (host) = 1 when the Cholesky factorisation of G - (tau + delta) I runs to
 * completion in FP64, delta = 2 (n + 4) 2^-53 trace(G): then every eigenvalue of G exceeds tau (delta
 * covers the factorisation's backward error, gamma_{n+1} |L||L^T|, bounded through the trace).
 * *above = 0 when a pivot is <= 0 or not a number: no certificate, which does not prove the converse
 * (an eigenvalue within delta of tau). BHT-l2r gives a certified interior node the identity as its
 * basis and skips its products. n <= 4096 (BHT_ECAPACITY), tau finite and >= 0 (else BHT_EINVAL).
 * Synchronises `stream`. */
bht_status bht_eig_min_above(const double* G, int64_t n, double tau, int32_t* above, void* stream);

/* Getters. Ranks: ranks[0] = items in the accumulation, ranks[i] = rank of
 * node i (breadth-first) for i = 1 .. 2d-2; `cap` is the length of `ranks`. */
bht_status bht_get_ranks(const bht_state* state, int64_t* ranks, int64_t cap);
bht_status bht_get_dims(const bht_state* state, int32_t* d, int64_t* dims, int64_t cap);
/* Copy core `node` (1 .. 2d-2) to host FP64 in the layout above; `cap` is the
 * capacity of `host_out` in elements; `numel` receives the element count. */
bht_status bht_get_core(const bht_state* state, int32_t node, double* host_out,
                        int64_t cap, int64_t* numel);
/* Copy root slices first .. first+count-1 to host FP64, [count][r_11][r_12]. */
bht_status bht_get_root(const bht_state* state, int64_t first, int64_t count,
                        double* host_out, int64_t cap);
/* Elements of all cores (denominator of the compression ratio, eq. compression_ratio). */
bht_status bht_num_elements(const bht_state* state, int64_t* cores_total);
bht_status bht_state_destroy(bht_state* state);

/* Device kernels launched by the calling thread's library calls since the
 * last reset (a plain counter kept by the host side of the library). */
bht_status bht_launch_count(int64_t* count, int32_t reset);

/* Kernels launched by the calling thread's compression calls (bht_l2r, ht_l2r, htrise_update) that
 * read the call's whole input batch, since the last reset: the number of passes over the data. */
bht_status bht_batch_reads(int64_t* count, int32_t reset);

/* Test of the timeout path (no counterpart in the paper): the next `launches` cooperative
 * tridiagonalisations of the node eigensolver that run on more than one CTA start with CTA 0
 * withholding its first grid-barrier arrival, and every wait of those launches gives up after
 * `wait_ms` milliseconds (1..65535). The waiting CTAs then set the call's device status word and
 * return, the context stays usable, and the library call that launched the eigensolve fails with
 * BHT_ETIMEOUT (htrise_update leaves its state as it was). launches = 0 disarms. Process-wide. */
bht_status bht_debug_withhold_barrier(int32_t launches, int32_t wait_ms);

/* Measured FMA throughput of the current GPU in TFLOP/s (2 flops per FMA) for dtype BHT_F64 or
 * BHT_F32: a launch of independent FMA chains on every SM, about 10 ms at the nominal rate, timed
 * with CUDA events on `stream` after a warm-up launch. This is the denominator of the ALU rooflines
 * of the FP64 node linear algebra and of the FP32 SIMT kernels (the paper has no counterpart).
 * Synchronises `stream`. */
bht_status bht_probe_fma_rate(int32_t dtype, double* tflops, void* stream);

/* Optional kernel timing. With bit c of class_mask set, every launch of
 * kernel class c made by the calling thread is bracketed by a CUDA event pair
 * recorded on its launch stream. bht_profile_read() waits for the recorded
 * events and returns, per class c < n (n >= 21), the summed durations in ms,
 * the launch counts and the algorithmic work of the timed launches (flops and
 * bytes the mathematics of each launch requires); reset != 0 clears them.
 * Any output pointer may be NULL. Class names come from bht_kernel_class_name(c). */
bht_status bht_profile_enable(uint32_t class_mask);
bht_status bht_profile_read(double* ms, int64_t* launches, double* flops, double* bytes, int32_t n,
                            int32_t reset);
const char* bht_kernel_class_name(int32_t cls);

/* ---------------------------------------------------------------------------------------------
 * Rank / expansion predictor (no counterpart in the paper). Parameters as one fp32 vector, flattened
 * W1 [hidden][f_in], b1 [hidden], W2 [hidden][hidden], b2 [hidden], W3 [2][hidden], b3 [2]; the library
 * keeps an FP32 master copy, Adam moments, the last gradient and a bf16 copy on the current device.
 * Forward: x~ = bf16(x); h1 = bf16(relu(bf16(W1) x~ + b1)); h2 = bf16(relu(bf16(W2) h1 + b2));
 * o = bf16(W3) h2 + b3 (FP32 accumulation); o0 = rank as a fraction of the node's residual dimension,
 * o1 = logit of "the batch expands the node". Loss: mean over the batch of (o0 - t0)^2 +
 * log(1 + exp(o1)) - t1 o1. Pointers may be host or device.
 * ------------------------------------------------------------------------------------------- */
bht_status bht_mlp_create(int32_t f_in, int32_t hidden, const float* params, bht_mlp** out);
bht_status bht_mlp_destroy(bht_mlp* net);
bht_status bht_mlp_num_params(const bht_mlp* net, int64_t* n);
/* Parameters (cap >= n) and, when grad_out is not NULL, the gradient of the last loss_grad call. */
bht_status bht_mlp_get_params(const bht_mlp* net, float* out, int64_t cap, float* grad_out);
/* out [B][2] = o for the inputs X [B][f_in]. */
bht_status bht_mlp_forward(const bht_mlp* net, const float* X, int64_t B, float* out, void* stream);
/* Loss of X [B][f_in] against targets T [B][2] into *loss (host, nullable); its gradient with
 * respect to the bf16 weights (straight through the rounding) is kept for bht_mlp_adam_step. */
bht_status bht_mlp_loss_grad(bht_mlp* net, const float* X, const float* T, int64_t B, double* loss, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the last gradient. */
bht_status bht_mlp_adam_step(bht_mlp* net, double lr, void* stream);
/* The predictor's 66 inputs for a node whose Gram matrix is G (c x c, FP64, symmetric positive
 * semidefinite, host or device): f[i] = log10(s_i / s_1), i < 64, for the descending singular values
 * of a Gaussian sketch of width 128 (-16 where there are none), f[64] = log10(tol / norm),
 * f[65] = log2(c) / 10. seed selects the sketch. */
bht_status bht_sketch_features(const double* G, int64_t c, double tol, double norm, uint64_t seed, float* feat,
                               void* stream);

const char* bht_last_error(void);
const char* bht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BHT_H_ */

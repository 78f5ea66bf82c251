// api.cu — host side of libbht: dimension tree, device state, orchestration
// of BHT-l2r (Algorithm 1) and HT-RISE (Algorithm 2), reconstruction
// (eq. htucker_reconstruction) and the C ABI of include/bht.h.
//
// Layout of a layer intermediate ("layer tensor"): item-major
// [N][I_1]..[I_m], one axis per node of the layer (eq.
// ht_index_set_construction with the batch appended, Section 3.1). The
// unfolding of axis j is the view [A][I_j][B], A = N * prod_{i<j} I_i,
// B = prod_{i>j} I_i; merging two children's axes into their parent's axis is
// a C-order reshape and moves no data.
#include <algorithm>
#include <exception>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bht.h"
#include "internal.cuh"

// ---------------------------------------------------------------------------
// errors, launch counter
// ---------------------------------------------------------------------------
namespace {
thread_local std::string g_err;
thread_local int64_t g_launches = 0;
// the device batch of the compression call running on this thread, and the kernels that read it whole
thread_local const void* g_batch = nullptr;
thread_local int64_t g_batch_reads = 0;

void note_read(const void* p) {
  if (p && p == g_batch) ++g_batch_reads;
}

// Marks the batch of one compression call for the read count, for the lifetime of the call.
struct BatchScope {
  explicit BatchScope(const void* p) { g_batch = p; }
  ~BatchScope() { g_batch = nullptr; }
};

struct Fail {
  bht_status st;
};

[[noreturn]] void fail(bht_status st, const std::string& msg) {
  g_err = msg;
  throw Fail{st};
}

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? BHT_ENOMEM : BHT_ECUDA,
         std::string(what) + ": " + cudaGetErrorString(e));
  }
}
}  // namespace

// ---------------------------------------------------------------------------
// optional per-launch CUDA-event profiler (per kernel class, per host thread)
// ---------------------------------------------------------------------------
namespace {
struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};
thread_local uint32_t g_prof_mask = 0;
thread_local std::vector<ProfRec> g_prof_pending;
thread_local std::vector<cudaEvent_t> g_prof_pool;
thread_local double g_prof_ms[bht::K_NUM_CLASSES] = {};
thread_local int64_t g_prof_n[bht::K_NUM_CLASSES] = {};
thread_local double g_prof_flops[bht::K_NUM_CLASSES] = {};
thread_local double g_prof_bytes[bht::K_NUM_CLASSES] = {};

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_resolve() {
  for (auto& r : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_prof_ms[r.cls] += ms;
      g_prof_n[r.cls] += 1;
    } else {
      cudaGetLastError();
    }
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_pending.clear();
}

// The thread-local counters of a worker thread (launches, per-class profile), carried back to the
// thread that made the library call.
struct ThreadCounters {
  int64_t launches = 0, batch_reads = 0;
  double ms[bht::K_NUM_CLASSES] = {}, flops[bht::K_NUM_CLASSES] = {}, bytes[bht::K_NUM_CLASSES] = {};
  int64_t n[bht::K_NUM_CLASSES] = {};
};

ThreadCounters take_thread_counters() {
  prof_resolve();
  ThreadCounters c;
  c.launches = g_launches;
  g_launches = 0;
  c.batch_reads = g_batch_reads;
  g_batch_reads = 0;
  for (int i = 0; i < bht::K_NUM_CLASSES; ++i) {
    c.ms[i] = g_prof_ms[i];
    c.n[i] = g_prof_n[i];
    c.flops[i] = g_prof_flops[i];
    c.bytes[i] = g_prof_bytes[i];
    g_prof_ms[i] = g_prof_flops[i] = g_prof_bytes[i] = 0.0;
    g_prof_n[i] = 0;
  }
  return c;
}

void add_thread_counters(const ThreadCounters& c) {
  g_launches += c.launches;
  g_batch_reads += c.batch_reads;
  for (int i = 0; i < bht::K_NUM_CLASSES; ++i) {
    g_prof_ms[i] += c.ms[i];
    g_prof_n[i] += c.n[i];
    g_prof_flops[i] += c.flops[i];
    g_prof_bytes[i] += c.bytes[i];
  }
}
}  // namespace

namespace bht {
void note_launch(int n) { g_launches += n; }
void set_last_error(const char* msg) { g_err = msg; }

cudaError_t allow_max_smem(const void* func) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& d : done)
    if (d.first == func && d.second == dev) return cudaSuccess;
  int cap = 0;
  e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  // the cap covers the dynamic part only: the opt-in maximum less the kernel's static shared memory
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, cap - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.push_back({func, dev});
  return e;
}

const char* kernel_class_name(int cls) {
  static const char* names[K_NUM_CLASSES] = {"gram_f64",       "ttm_f64",        "eig_tridiag_f64", "eig_bisect_f64",
                                             "gemm_f64",       "norm",           "copy",            "ttm_tc",
                                             "gram_f32",       "eig_vec_f64",    "eig_back_f64",    "ttm_f32",
                                             "house_f64",      "mlp",            "prep",            "other",
                                             "pair_proj",      "pair_gram",      "spd_test_f64",   "tri_proj",       "ritz_small"};
  return (cls >= 0 && cls < K_NUM_CLASSES) ? names[cls] : "?";
}

ProfScope::ProfScope(int cls, cudaStream_t s, double flops, double bytes)
    : cls_(cls), s_(s), on_(((g_prof_mask >> cls) & 1u) != 0) {
  if (on_) {
    g_prof_flops[cls] += flops;
    g_prof_bytes[cls] += bytes;
    e0_ = prof_event();
    cudaEventRecord(e0_, s_);
  }
}

ProfScope::~ProfScope() {
  if (on_) {
    cudaEvent_t e1 = prof_event();
    cudaEventRecord(e1, s_);
    g_prof_pending.push_back({cls_, e0_, e1});
  }
}
}  // namespace bht

using namespace bht;

// ---------------------------------------------------------------------------
// dimension tree (Section 2.3, Fig. 2)
// ---------------------------------------------------------------------------
struct TNode {
  int id = 0, layer = 0, parent = -1, slot = -1;
  int child[2] = {-1, -1};
  int mode = -1;              // leaf: its mode
  int first = 0, count = 0;   // modes covered: first .. first+count-1
  bool leaf() const { return child[0] < 0; }
};

struct bht_tree {
  int d = 0;
  std::vector<int64_t> dims;
  std::vector<TNode> nodes;                 // breadth-first, root = 0
  std::vector<std::vector<int>> layers;     // node ids per layer, left to right
  int p = 0;
  std::vector<int> leaf_of_mode;
};

static void build_tree(bht_tree& t, int d, const int64_t* dims) {
  t.d = d;
  t.dims.assign(dims, dims + d);
  t.nodes.clear();
  t.layers.clear();
  TNode root;
  root.id = 0;
  root.first = 0;
  root.count = d;
  t.nodes.push_back(root);
  std::vector<int> frontier = {0};
  while (!frontier.empty()) {
    t.layers.push_back(frontier);
    std::vector<int> next;
    for (int id : frontier) {
      const int m = t.nodes[id].count;
      if (m == 1) {
        t.nodes[id].mode = t.nodes[id].first;
        continue;
      }
      const int h = (m + 1) / 2;  // the first successor takes ceil(m/2) modes
      for (int slot = 0; slot < 2; ++slot) {
        TNode c;
        c.id = (int)t.nodes.size();
        c.layer = t.nodes[id].layer + 1;
        c.parent = id;
        c.slot = slot;
        c.first = t.nodes[id].first + (slot ? h : 0);
        c.count = slot ? m - h : h;
        t.nodes[id].child[slot] = c.id;
        t.nodes.push_back(c);
        next.push_back(c.id);
      }
    }
    frontier = next;
  }
  t.p = (int)t.layers.size() - 1;
  t.leaf_of_mode.assign(d, -1);
  for (auto& nd : t.nodes)
    if (nd.leaf()) t.leaf_of_mode[nd.mode] = nd.id;
}

// ---------------------------------------------------------------------------
// device memory helpers (stream-ordered pool allocations)
// ---------------------------------------------------------------------------
namespace {

// Stream-ordered allocations from the device's default pool. The pool keeps what it has
// grown to (release threshold raised once per device, for this process only): the working
// buffers of one update are allocated and freed many times per call, and a pool that hands
// memory back at every synchronisation would map it again each time.
void keep_pool(int dev) {
  static std::mutex mu;
  static bool done[64] = {};
  if (dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

void* dalloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) keep_pool(dev);
  void* p = nullptr;
  ck(cudaMallocAsync(&p, bytes, s), "cudaMallocAsync");
  return p;
}
void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

struct DBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t bytes, cudaStream_t st) : p(dalloc(bytes, st)), s(st) {}
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), s(o.s) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      dfree(p, s);
      p = o.p;
      s = o.s;
      o.p = nullptr;
    }
    return *this;
  }
  ~DBuf() { dfree(p, s); }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t dtype_size(int dt) { return dt == BHT_F64 ? 8 : 4; }

}  // namespace

// ---------------------------------------------------------------------------
// state
// ---------------------------------------------------------------------------
struct bht_state {
  bht_tree tree;
  int precision = BHT_PREC_FP64;
  int budget = BHT_BUDGET_UNIFORM;  // default node-wise budget of htrise_update
  std::vector<int64_t> rank;    // per node id; rank[0] unused
  std::vector<double*> U;       // per node id: orthonormal matrix form [rows][rank], FP64, device
  std::vector<double*> Q;       // per node id: orthonormal complement of U in R^rows, [rows][rows - rank]
  // per node id: the basis U[id] when it is the identity of R^rows (a node whose truncation keeps every
  // direction), else null. A product with it leaves the tensor as it is and is not launched. Cleared
  // when the node's basis is replaced (a padded or expanded core is no longer the identity).
  std::vector<const double*> ident;
  double* root = nullptr;       // [root_cap][r11][r12], FP64, device
  int64_t root_cap = 0;
  int64_t n_items = 0;
  int* d_status = nullptr;      // device status word of bounded waits
  bool plain = false;           // plain HT of one tensor (n_1..n_d, N): the batch is a leaf, not the root's
  // Tensor-core weight planes (kind 1) and FP32 copies [S1 + S2][T] for the SIMT kernel (kind 2, the
  // basis read as M(s, t) = U[s ms + t mt]) of committed cores and their complements, prepared once:
  // the cores of a skipped update do not change. Keyed by the core pointers; entries go when a core is
  // released.
  struct TcWeights {
    const double* U;
    const double* Q;
    int64_t S1, S2, T, kv;
    int transpose;
    float* W;
    int64_t ms = 0, mt = 0;
  };
  mutable std::vector<TcWeights> wcache;
  mutable std::mutex wmu;
  // pinned host slots the skip test of Algorithm 2 reads back into (two, for the pipelined stream of
  // batches): ||Y||^2, ||C||^2, the projection error and the status word of the bounded waits
  double* pinned = nullptr;

  int64_t rows(int id) const {  // alpha of eq. compute_residual; n for a leaf
    const TNode& nd = tree.nodes[id];
    if (nd.leaf()) return tree.dims[nd.mode];
    return rank[nd.child[0]] * rank[nd.child[1]];
  }
  int64_t r11() const { return rank[tree.nodes[0].child[0]]; }
  int64_t r12() const { return rank[tree.nodes[0].child[1]]; }
};

// Rank / expansion predictor: FP32 master parameters, Adam moments, the last gradient and the bf16
// copy the kernels read, all on the device where it was created. Layout of the flat parameter
// vector: W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [2][H], b3 [2].
struct bht_mlp {
  int f_in = 66, hidden = 128;
  int64_t P = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
  __nv_bfloat16* wq = nullptr;
  int64_t steps = 0;
  int64_t oW1() const { return 0; }
  int64_t ob1() const { return (int64_t)hidden * f_in; }
  int64_t oW2() const { return ob1() + hidden; }
  int64_t ob2() const { return oW2() + (int64_t)hidden * hidden; }
  int64_t oW3() const { return ob2() + hidden; }
  int64_t ob3() const { return oW3() + 2 * (int64_t)hidden; }
};

namespace {

// ---------------------------------------------------------------------------
// layer tensors
// ---------------------------------------------------------------------------
struct LTensor {
  const void* ptr = nullptr;
  int dtype = BHT_F64;
  int64_t N = 0;
  std::vector<int64_t> dims;   // per axis
  std::vector<int> node;       // node id carried by each axis
  DBuf own;                    // owns ptr when the library created it

  int64_t numel() const {
    int64_t n = N;
    for (auto v : dims) n *= v;
    return n;
  }
  LTensor view_copy() const {  // a non-owning view of the same data
    LTensor v;
    v.ptr = ptr;
    v.dtype = dtype;
    v.N = N;
    v.dims = dims;
    v.node = node;
    return v;
  }
  int axis_of(int id) const {
    for (size_t i = 0; i < node.size(); ++i)
      if (node[i] == id) return (int)i;
    fail(BHT_EINVAL, "internal: node not on an axis");
  }
  void view(int axis, int64_t& A, int64_t& I, int64_t& B) const {
    A = N;
    for (int i = 0; i < axis; ++i) A *= dims[i];
    I = dims[axis];
    B = 1;
    for (size_t i = axis + 1; i < dims.size(); ++i) B *= dims[i];
  }
};

LTensor input_tensor(const bht_tree& t, const void* Y, int dtype, int64_t N) {
  LTensor C;
  C.ptr = Y;
  C.dtype = dtype;
  C.N = N;
  C.dims = t.dims;
  for (int m = 0; m < t.d; ++m) C.node.push_back(t.leaf_of_mode[m]);
  return C;
}

// Merge the axes of layer+1 into the index set of `layer` (eq. ht_index_set_construction):
// a transfer node's two successors are adjacent axes, merged in C-order.
void reshape_to_layer(const bht_tree& t, LTensor& C, int layer) {
  std::vector<int64_t> dims;
  std::vector<int> node;
  size_t pos = 0;
  for (int id : t.layers[layer]) {
    const TNode& nd = t.nodes[id];
    if (nd.leaf()) {
      if (pos >= C.node.size() || C.node[pos] != id) fail(BHT_EINVAL, "internal: reshape (leaf)");
      dims.push_back(C.dims[pos]);
      pos += 1;
    } else {
      if (pos + 1 >= C.node.size() + 1 || C.node[pos] != nd.child[0] || C.node[pos + 1] != nd.child[1])
        fail(BHT_EINVAL, "internal: reshape (transfer)");
      dims.push_back(C.dims[pos] * C.dims[pos + 1]);
      pos += 2;
    }
    node.push_back(id);
  }
  C.dims = dims;
  C.node = node;
}

// Order of contractions over several axes of one layer minimising FP work.
// ops: (axis, new size). Exhaustive for <= 6 operations.
std::vector<int> best_order(const std::vector<int64_t>& dims, const std::vector<std::pair<int, int64_t>>& ops) {
  std::vector<int> perm(ops.size());
  for (size_t i = 0; i < perm.size(); ++i) perm[i] = (int)i;
  auto cost = [&](const std::vector<int>& pr) {
    std::vector<double> d(dims.begin(), dims.end());
    double c = 0.0;
    for (int k : pr) {
      double prod = 1.0;
      for (size_t i = 0; i < d.size(); ++i) prod *= d[i];
      c += prod * (double)ops[k].second;  // 2 * I * S * rest, up to the factor 2
      d[ops[k].first] = (double)ops[k].second;
    }
    return c;
  };
  if (ops.size() <= 1) return perm;
  std::vector<int> best = perm;
  double bc = cost(perm);
  if (ops.size() <= 6) {
    while (std::next_permutation(perm.begin(), perm.end())) {
      const double c = cost(perm);
      if (c < bc) {
        bc = c;
        best = perm;
      }
    }
  }
  return best;
}

// ---------------------------------------------------------------------------
// Arithmetic of one call
//   FP64 : every contraction, Gram, norm and eigensolve in FP64.
//   mixed: full-data contractions of an innermost axis on tcgen05 tensor cores
//          (split TF32, FP32 accumulation), other contractions in FP32 SIMT,
//          Grams with FP32 products promoted to FP64 every 16 columns; node
//          eigensolves, orthogonalisation and norms in FP64 (the tensor-core
//          kernel folds ||Y||^2 from FP32 partial sums of 16 squares). At tight
//          tolerances (eps_rel < 1e-3) the Grams stay FP64 and ||Y||^2 is
//          summed in FP64 from the data.
// ---------------------------------------------------------------------------
struct Arith {
  bool mixed = false;
  bool tight = false;
  // the two-mode FP32 SIMT passes of small leaves (pair.cu) may replace the per-mode products: their
  // bases are rounded to FP32, which moves the projection energies of the skip test by about 2e-8 of
  // ||Y||^2 (measured on the sensor stream), below 0.1 % of eps^2 ||Y||^2 for eps_rel >= 5e-3
  bool pairs = false;
  int* d_status = nullptr;
};

void gram_any(const LTensor& C, int axis, double* G, const Arith& ar, cudaStream_t s) {
  int64_t A, I, B;
  C.view(axis, A, I, B);
  note_read(C.ptr);
  ck(cudaMemsetAsync(G, 0, sizeof(double) * I * I, s), "memset gram");
  if (C.dtype == BHT_F32 && ar.mixed && !ar.tight)
    ck(launch_gram_f32(static_cast<const float*>(C.ptr), G, A, I, B, s), "gram");
  else if (C.dtype == BHT_F32)
    ck(launch_gram_f64<float>(static_cast<const float*>(C.ptr), G, A, I, B, s), "gram");
  else
    ck(launch_gram_f64<double>(static_cast<const double*>(C.ptr), G, A, I, B, s), "gram");
}

// Weights of a committed core (U [T][S1] read transposed, and Q [T][S2] when given) for the tensor-core
// mode product: prepared on first use for the state, then reused until the core is released.
const float* state_weights(const bht_state* st, const double* U, int64_t S1, const double* Q, int64_t S2, int64_t T,
                           int64_t kv, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(st->wmu);
  for (const auto& w : st->wcache)
    if (w.U == U && w.Q == Q && w.S1 == S1 && w.S2 == S2 && w.T == T && w.kv == kv && w.transpose == 1) return w.W;
  float* W = static_cast<float*>(dalloc(ttm_tc_weights_bytes(T, S1 + S2), s));
  try {
    ck(launch_prep_tc_weights2(U, S1, S1, Q, S2, S2, T, true, W, 2, s, kv), "tc weights");
  } catch (...) {
    dfree(W, s);
    throw;
  }
  st->wcache.push_back({U, Q, S1, S2, T, kv, 1, W});
  return W;
}

// FP32 copy [S1 + S2][T] of a committed core (M(s, t) = U[s ms + t mt], s < S1) followed by its
// complement Q [T][S2] read transposed, for the FP32 SIMT mode product: made on first use for the
// state, then reused until the core is released.
const float* state_basis32(const bht_state* st, const double* U, int64_t ms, int64_t mt, int64_t S1, const double* Q,
                           int64_t S2, int64_t T, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(st->wmu);
  for (const auto& w : st->wcache)
    if (w.transpose == 2 && w.U == U && w.Q == Q && w.S1 == S1 && w.S2 == S2 && w.T == T && w.ms == ms && w.mt == mt)
      return w.W;
  float* W = static_cast<float*>(dalloc(sizeof(float) * (size_t)std::max<int64_t>((S1 + S2) * T, 1), s));
  try {
    ck(launch_cast_matrix(U, ms, mt, S1, T, W, s), "basis to FP32");
    if (Q && S2 > 0) ck(launch_cast_matrix(Q, 1, S2, S2, T, W + S1 * T, s), "complement to FP32");
  } catch (...) {
    dfree(W, s);
    throw;
  }
  bht_state::TcWeights e{U, Q, S1, S2, T, -1, 2, W};
  e.ms = ms;
  e.mt = mt;
  st->wcache.push_back(e);
  return W;
}

// Drop the cached weights that read the core or complement p (before p is released).
void purge_weights(const bht_state* st, const double* p, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(st->wmu);
  // every earlier use was in a call that has finished; later work on s is ordered after the release
  auto& v = st->wcache;
  for (auto it = v.begin(); it != v.end();) {
    if (it->U == p || it->Q == p) {
      dfree(it->W, s);
      it = v.erase(it);
    } else {
      ++it;
    }
  }
}

// Mode product of axis `axis`: the axis (size T) becomes size S, new(s) = sum_t M(s, t) old(t),
// M(s, t) = U[s * ms + t * mt] (projection: U [T][S], ms = 1, mt = S; expansion: U [S][T], ms = T, mt = 1).
// rotate: only for the innermost axis, the new axis moves to the front (right after the items).
// norm_in (nullable, device double): ||C||^2 added in FP64 when the tensor-core kernel runs.
// k_valid >= 0: the axis is zero padded beyond its first k_valid entries (the basis has k_valid rows);
// only the tensor-core kernel takes such an axis.
LTensor ttm_any(const LTensor& C, int axis, const double* U, int64_t ms, int64_t mt, int64_t S, bool rotate,
                const Arith& ar, cudaStream_t s, double* norm_in = nullptr, bool* used_norm = nullptr,
                int64_t k_valid = -1, const bht_state* cache = nullptr) {
  int64_t A, T, B;
  C.view(axis, A, T, B);
  if (rotate && B != 1) fail(BHT_EINVAL, "internal: rotation of a non-innermost axis");
  note_read(C.ptr);
  LTensor out;
  out.N = C.N;
  out.dims = C.dims;
  out.node = C.node;
  out.dims[axis] = S;
  if (rotate) {  // new axis in front: [N][S][other axes in order]
    std::rotate(out.dims.begin(), out.dims.begin() + axis, out.dims.begin() + axis + 1);
    std::rotate(out.node.begin(), out.node.begin() + axis, out.node.begin() + axis + 1);
  }
  const int64_t R2 = rotate ? A / C.N : 1;  // rows per item behind the new axis
  if (used_norm) *used_norm = false;
  if (!ar.mixed) {
    if (rotate) fail(BHT_EINVAL, "internal: rotation in the FP64 form");
    out.dtype = BHT_F64;
    out.own = DBuf(sizeof(double) * (size_t)std::max<int64_t>(out.numel(), 1), s);
    out.ptr = out.own.p;
    if (C.dtype == BHT_F32)
      ck(launch_ttm_f64<float, double>(static_cast<const float*>(C.ptr), out.own.as<double>(), U, ms, mt, A, T, B,
                                       S, s),
         "ttm");
    else
      ck(launch_ttm_f64<double, double>(static_cast<const double*>(C.ptr), out.own.as<double>(), U, ms, mt, A, T, B,
                                        S, s),
         "ttm");
    return out;
  }
  out.dtype = BHT_F32;
  out.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(out.numel(), 1), s);
  out.ptr = out.own.p;
  const int nb = 2;  // the basis enters as TF32 plus its TF32 remainder: no rounding bias in any norm
  const bool aligned = (reinterpret_cast<uintptr_t>(C.ptr) & 15) == 0;
  if (B == 1 && C.dtype == BHT_F32 && aligned && ttm_tc_supported(T, S, nb)) {
    // W[s][t] = M(s, t): projection reads U transposed (ldu = S), expansion reads U as is (ldu = T)
    const bool transpose = (ms == 1);
    DBuf Wb;
    const float* W = nullptr;
    if (cache && transpose) {
      W = state_weights(cache, U, S, nullptr, 0, T, k_valid, s);
    } else {
      Wb = DBuf(ttm_tc_weights_bytes(T, S), s);
      ck(launch_prep_tc_weights2(U, S, transpose ? S : (k_valid >= 0 ? k_valid : T), nullptr, 0, 1, T, transpose,
                                 Wb.as<float>(), nb, s, k_valid),
         "tc weights");
      W = Wb.as<float>();
    }
    ck(launch_ttm_tc(static_cast<const float*>(C.ptr), A, T, W, S, nb, out.own.as<float>(), R2, norm_in, nullptr,
                     ar.d_status, s),
       "tensor-core mode product");
    if (used_norm) *used_norm = norm_in != nullptr;
    return out;
  }
  if (k_valid >= 0) fail(BHT_EINVAL, "internal: padded axis outside the tensor-core kernel");
  // the basis enters the FP32 SIMT kernel as an FP32 copy [S][T] (the state's, for a committed core)
  DBuf M32b;
  const float* M32 = nullptr;
  if (cache) {
    M32 = state_basis32(cache, U, ms, mt, S, nullptr, 0, T, s);
  } else {
    M32b = DBuf(sizeof(float) * (size_t)std::max<int64_t>(S * T, 1), s);
    ck(launch_cast_matrix(U, ms, mt, S, T, M32b.as<float>(), s), "basis to FP32");
    M32 = M32b.as<float>();
  }
  if (C.dtype == BHT_F32)
    ck(launch_ttm_f32<float>(static_cast<const float*>(C.ptr), out.own.as<float>(), M32, T, 1, A, T, B, S, R2, s),
       "ttm");
  else
    ck(launch_ttm_f32<double>(static_cast<const double*>(C.ptr), out.own.as<float>(), M32, T, 1, A, T, B, S, R2, s),
       "ttm");
  return out;
}

// Mixed-path projection of one axis onto [U | Q] (U [T][r] the node basis, Q [T][c] its orthonormal
// complement): the r outputs on U are kept, the squares of the c outputs on Q (the energy of the part
// of C outside span(U) along this axis) are added to *resid without forming them. As [U | Q] is
// orthogonal, ||C||^2 = ||C x U^T||^2 + ||C x Q^T||^2 exactly; the sum of these residual energies over a
// full projection is the projection error of eq. relative_error_threshold, free of the cancellation
// in ||Y||^2 - ||C||^2.
LTensor ttm_proj_resid(const LTensor& C, int axis, const double* U, int64_t r, const double* Q, int64_t c,
                       bool rotate, const Arith& ar, cudaStream_t s, double* norm_in, bool* used_norm,
                       double* resid, int64_t k_valid = -1, const bht_state* cache = nullptr) {
  if (!ar.mixed || !resid || c <= 0)
    return ttm_any(C, axis, U, 1, r, r, rotate, ar, s, norm_in, used_norm, k_valid, cache);
  int64_t A, T, B;
  C.view(axis, A, T, B);
  if (rotate && B != 1) fail(BHT_EINVAL, "internal: rotation of a non-innermost axis");
  note_read(C.ptr);
  LTensor out;
  out.N = C.N;
  out.dims = C.dims;
  out.node = C.node;
  out.dims[axis] = r;
  if (rotate) {
    std::rotate(out.dims.begin(), out.dims.begin() + axis, out.dims.begin() + axis + 1);
    std::rotate(out.node.begin(), out.node.begin() + axis, out.node.begin() + axis + 1);
  }
  const int64_t R2 = rotate ? A / C.N : 1;
  if (used_norm) *used_norm = false;
  out.dtype = BHT_F32;
  out.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(out.numel(), 1), s);
  out.ptr = out.own.p;
  const int nb = 2;
  const bool aligned = (reinterpret_cast<uintptr_t>(C.ptr) & 15) == 0;
  if (B == 1 && C.dtype == BHT_F32 && aligned && ttm_tc_supported(T, r + c, nb)) {
    DBuf Wb;
    const float* W = nullptr;
    if (cache) {
      W = state_weights(cache, U, r, Q, c, T, k_valid, s);
    } else {
      Wb = DBuf(ttm_tc_weights_bytes(T, r + c), s);
      ck(launch_prep_tc_weights2(U, r, r, Q, c, c, T, true, Wb.as<float>(), nb, s, k_valid), "tc weights");
      W = Wb.as<float>();
    }
    ck(launch_ttm_tc_resid(static_cast<const float*>(C.ptr), A, T, W, r + c, r, nb, out.own.as<float>(), R2, norm_in,
                           nullptr, resid, ar.d_status, s),
       "tensor-core mode product");
    if (used_norm) *used_norm = norm_in != nullptr;
    return out;
  }
  if (k_valid >= 0) fail(BHT_EINVAL, "internal: padded axis outside the tensor-core kernel");
  // FP32 SIMT on [U | Q] cast to fp32 [r + c][T] (the state's copy, for a committed core)
  DBuf M32b;
  const float* M32 = nullptr;
  if (cache) {
    M32 = state_basis32(cache, U, 1, r, r, Q, c, T, s);
  } else {
    M32b = DBuf(sizeof(float) * (size_t)std::max<int64_t>((r + c) * T, 1), s);
    ck(launch_cast_matrix(U, 1, r, r, T, M32b.as<float>(), s), "basis to FP32");
    ck(launch_cast_matrix(Q, 1, c, c, T, M32b.as<float>() + r * T, s), "complement to FP32");
    M32 = M32b.as<float>();
  }
  if (C.dtype == BHT_F32)
    ck(launch_ttm_f32_resid<float>(static_cast<const float*>(C.ptr), out.own.as<float>(), M32, T, 1, A, T, B, r + c,
                                   r, R2, resid, s),
       "ttm");
  else
    ck(launch_ttm_f32_resid<double>(static_cast<const double*>(C.ptr), out.own.as<float>(), M32, T, 1, A, T, B,
                                    r + c, r, R2, resid, s),
       "ttm");
  return out;
}

// The axis `ax` of an fp32 tensor moved innermost and zero padded to a multiple of four entries (rows
// the tensor-core kernel's TMA reads in 16-byte steps). The last axis of the result carries the node of
// `ax` with the padded size; *k_valid receives its true size.
LTensor move_axis_innermost(const LTensor& C, int ax, int64_t* k_valid, cudaStream_t s) {
  int64_t A, T, B;
  C.view(ax, A, T, B);
  note_read(C.ptr);
  const int64_t Tp = (T + 3) / 4 * 4;
  LTensor out;
  out.dtype = BHT_F32;
  out.N = C.N;
  for (size_t i = 0; i < C.dims.size(); ++i)
    if ((int)i != ax) {
      out.dims.push_back(C.dims[i]);
      out.node.push_back(C.node[i]);
    }
  out.dims.push_back(Tp);
  out.node.push_back(C.node[ax]);
  out.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(A * B * Tp, 1), s);
  out.ptr = out.own.p;
  ck(launch_transpose_pad(static_cast<const float*>(C.ptr), out.own.as<float>(), A, T, B, Tp, s), "axis innermost");
  *k_valid = T;
  return out;
}

// Reorder the axes of C to `order` (node ids), moving data only when the order differs.
void restore_axis_order(LTensor& C, const std::vector<int>& order, cudaStream_t s) {
  const int d = (int)order.size();
  std::vector<int> perm(d);
  bool same = true;
  for (int k = 0; k < d; ++k) {
    perm[k] = C.axis_of(order[k]);
    same = same && perm[k] == k;
  }
  if (same) return;
  LTensor out;
  out.dtype = C.dtype;
  out.N = C.N;
  out.node = order;
  for (int k = 0; k < d; ++k) out.dims.push_back(C.dims[perm[k]]);
  out.own = DBuf(dtype_size(C.dtype) * (size_t)std::max<int64_t>(C.numel(), 1), s);
  out.ptr = out.own.p;
  ck(launch_permute_items(C.ptr, C.dtype, C.N, d, C.dims.data(), perm.data(), out.own.p, s), "axis order");
  C = std::move(out);
}

// Mixed form of a layer's projections on the tensor cores: each listed axis, from the innermost
// outward, is contracted as the innermost axis (moved there, zero padded, when it is not a
// multiple-of-four innermost axis) with the new axis rotated to the front; when every axis of the
// layer is listed the rotations alone restore the order, otherwise one permutation does. With Qs
// and resid, each axis is projected onto [U | Q] and the complement energy is added to *resid.
LTensor project_layer_tc(LTensor C, const std::vector<int>& ids, const std::vector<const double*>& Us,
                         const std::vector<int64_t>& rs, const std::vector<const double*>* Qs,
                         const std::vector<int64_t>* qcs, double* resid, const Arith& ar, cudaStream_t s,
                         const bht_state* cache = nullptr) {
  const std::vector<int> order0 = C.node;
  std::vector<int> ks(ids.size());
  for (size_t k = 0; k < ks.size(); ++k) ks[k] = (int)k;
  std::sort(ks.begin(), ks.end(), [&](int a, int b) { return C.axis_of(ids[a]) > C.axis_of(ids[b]); });
  for (int k : ks) {
    int ax = C.axis_of(ids[k]);
    int64_t A, T, B, kv = -1;
    C.view(ax, A, T, B);
    if (B != 1 || T % 4 != 0 || (reinterpret_cast<uintptr_t>(C.ptr) & 15) != 0) {
      C = move_axis_innermost(C, ax, &kv, s);
      ax = (int)C.dims.size() - 1;
    }
    LTensor nxt = (resid && Qs) ? ttm_proj_resid(C, ax, Us[k], rs[k], (*Qs)[k], (*qcs)[k], true, ar, s, nullptr, nullptr,
                                                 resid, kv, cache)
                                : ttm_any(C, ax, Us[k], 1, rs[k], rs[k], true, ar, s, nullptr, nullptr, kv, cache);
    C = std::move(nxt);
  }
  restore_axis_order(C, order0, s);
  return C;
}

// Whether every product of a layer is small enough (at most about a GFLOP, 2 numel S with S the new
// size) for the FP32 SIMT kernel in place: there the tensor cores' transposes and permutations cost
// more than the product. BHT-l2r, Step 1 and Step 3 of HT-RISE take the same rule, so that a batch is
// encoded in the same arithmetic by each of them.
bool small_products(const LTensor& C, const std::vector<int64_t>& sizes) {
  double mx = 0.0;
  for (int64_t v : sizes) mx = std::max(mx, 2.0 * (double)C.numel() * (double)v);
  return C.dtype == BHT_F32 && mx <= 1e9;
}

// Project a layer's axes onto bases (C x_j U_j^T), U_j = [rows_j][r_j], cheapest order first.
LTensor project_layer(LTensor C, const std::vector<int>& ids, const std::vector<const double*>& Us,
                      const std::vector<int64_t>& rs, const Arith& ar, cudaStream_t s) {
  if (ar.mixed && !ar.tight && C.dtype == BHT_F32 && !ids.empty() && !small_products(C, rs))
    return project_layer_tc(std::move(C), ids, Us, rs, nullptr, nullptr, nullptr, ar, s);
  std::vector<std::pair<int, int64_t>> ops;
  for (size_t k = 0; k < ids.size(); ++k) ops.push_back({C.axis_of(ids[k]), rs[k]});
  for (int k : best_order(C.dims, ops)) {
    LTensor nxt = ttm_any(C, C.axis_of(ids[k]), Us[k], 1, rs[k], rs[k], false, ar, s);
    C = std::move(nxt);
  }
  return C;
}

struct EigOut {
  DBuf work, lam;
  int64_t n = 0;
  int64_t computed = 0;          // eigenvalues known: descending indices [0, computed)
  double trace = 0.0;            // trace of the matrix (= sum of the tridiagonal's diagonal)
  std::vector<double> h_lam;     // host copy of lam[0, computed)
  std::vector<double> h_diag;
};

// Stage 1a of the eigensolver: tridiagonalise the symmetric FP64 matrix G (destroyed) and start the
// copy of the tridiagonal's diagonal (its sum is the trace) to the host.
void eig_tridiag64(double* G, int64_t n, EigOut& out, int* d_status, cudaStream_t s) {
  out.n = n;
  out.computed = 0;
  out.lam = DBuf(sizeof(double) * n, s);
  out.work = DBuf(eig_workspace_bytes(n), s);
  ck(launch_eig_tridiag(G, n, out.work.p, d_status, s), "tridiagonalisation");
  out.h_diag.resize(n);
  ck(cudaMemcpyAsync(out.h_diag.data(), eig_tridiag_diagonal(out.work.p, n), sizeof(double) * n,
                     cudaMemcpyDeviceToHost, s),
     "D2H diagonal");
}

// Stage 1 complete: every eigenvalue (for the small nodes and the explicit entry point).
void eig_values64(double* G, int64_t n, EigOut& out, int* d_status, cudaStream_t s) {
  eig_tridiag64(G, n, out, d_status, s);
  ck(launch_eig_bisect(n, out.work.p, out.lam.as<double>(), 0, n, s), "eigenvalues");
  out.computed = n;
}

// The tail rule of eq. ht_leaf_svd / eq. svd_on_residual on all n eigenvalues lam (decreasing) of a
// Gram matrix of trace tr: the smallest r >= rmin whose discarded energy tr - sum_{i<r} lam_i is at most
// eps_nw2 (r = n discards nothing), capped at rmax.
int64_t tail_rank(const double* lam, int64_t n, double tr, double eps_nw2, int64_t rmin, int64_t rmax) {
  rmax = std::min(rmax, n);
  double kept = 0.0;
  for (int64_t r = 0; r <= n; ++r) {
    if (r >= rmin) {
      const double tail = (r == n) ? 0.0 : std::max(tr - kept, 0.0);
      if (tail <= eps_nw2 || r >= rmax) return std::min(r, rmax);
    }
    if (r < n) kept += std::max(lam[r], 0.0);
  }
  return rmax;
}

// Truncation rank of eq. ht_leaf_svd / eq. svd_on_residual from the largest eigenvalues only: the
// discarded energy after r kept values is trace - sum_{i<r} lam_i, so eigenvalues are bisected from the
// top, in chunks that double, until some r >= rmin meets tail <= eps_nw2 (or all are known).
// Called after the tridiagonalisation has finished (the stream was synchronised).
int64_t eig_rank64(EigOut& eo, double eps_nw2, int64_t rmin, int64_t rmax, cudaStream_t s,
                   double trace = std::nan("")) {
  const int64_t n = eo.n;
  double tr = 0.0;
  for (double v : eo.h_diag) tr += v;
  if (std::isfinite(trace)) tr = trace;  // the trace of the Gram matrix itself, when the caller has it
  eo.trace = tr;
  rmax = std::min(rmax, n);
  // every eigenvalue in one launch: a Sturm sweep is latency-bound, so fewer eigenvalues do not cost less
  int64_t want = n;
  while (true) {
    if (want > eo.computed) {
      ck(launch_eig_bisect(n, eo.work.p, eo.lam.as<double>(), eo.computed, want, s), "eigenvalues");
      eo.h_lam.resize(want);
      ck(cudaMemcpyAsync(eo.h_lam.data() + eo.computed, eo.lam.as<double>() + eo.computed,
                         sizeof(double) * (want - eo.computed), cudaMemcpyDeviceToHost, s),
         "D2H eigenvalues");
      ck(cudaStreamSynchronize(s), "sync");
      eo.computed = want;
    }
    // smallest r >= rmin with tail(r) <= eps_nw2 among r <= computed; tail(n) = 0 when all are known
    double kept = 0.0;
    for (int64_t r = 0; r <= eo.computed; ++r) {
      if (r >= rmin) {
        const double tail = (r == n) ? 0.0 : std::max(tr - kept, 0.0);
        if (tail <= eps_nw2 || r >= rmax) return std::min(r, rmax);
      }
      if (r < eo.computed) kept += std::max(eo.h_lam[r], 0.0);
    }
    if (eo.computed >= n) return std::min(n, rmax);
    want = std::min<int64_t>(n, 2 * eo.computed);
  }
}

// X (rows x r) <- X (3I - X^T X) / 2: Newton-Schulz orthonormalisation of nearly orthonormal
// columns (an orthonormality error e becomes about 3e^2/4 per step).
void newton_schulz(double* X, int64_t rows, int64_t r, cudaStream_t s, int iters = 1) {
  if (r <= 0) return;
  DBuf S(sizeof(double) * r * r, s), T(sizeof(double) * rows * r, s);
  for (int it = 0; it < iters; ++it) {
    ck(launch_gemm_f64(r, r, rows, -0.5, X, 1, r, X, r, 1, 0.0, S.as<double>(), r, 1, s), "X^T X");
    ck(launch_add_diag(S.as<double>(), r, 1.5, s), "1.5 I");
    ck(launch_gemm_f64(rows, r, r, 1.0, X, r, 1, S.as<double>(), r, 1, 0.0, T.as<double>(), r, 1, s), "X S");
    ck(cudaMemcpyAsync(X, T.p, sizeof(double) * rows * r, cudaMemcpyDeviceToDevice, s), "copy");
  }
}

double sqnorm_of(const void* x, int dtype, int64_t n, double* d_acc, cudaStream_t s);

// Estimate of ||X^T X - I||_2 for X (rows x r): four power steps on E = X^T X - I from a
// pseudo-random start, each two matrix-vector products (the ratio of the last two iterates). For
// r <= 64, ||E||_F itself (an upper bound of ||E||_2) from E formed in one product: three launches
// instead of a dozen.
double orth_error(const double* X, int64_t rows, int64_t r, cudaStream_t s) {
  if (r <= 0) return 0.0;
  if (r <= 64) {
    DBuf E(sizeof(double) * r * r, s), acc(sizeof(double), s);
    ck(launch_gemm_f64(r, r, rows, 1.0, X, 1, r, X, r, 1, 0.0, E.as<double>(), r, 1, s), "X^T X");
    ck(launch_add_diag(E.as<double>(), r, -1.0, s), "- I");
    sqnorm_of(E.p, BHT_F64, r * r, acc.as<double>(), s);
    double h = 0.0;
    ck(cudaMemcpyAsync(&h, acc.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H probe");
    ck(cudaStreamSynchronize(s), "sync");
    return std::sqrt(h);
  }
  DBuf v(sizeof(double) * 2 * r, s), y(sizeof(double) * rows, s), acc(sizeof(double) * 2, s);
  double* x = v.as<double>();
  double* z = x + r;
  ck(launch_fill_uniform(x, r, 0x6f727468ull, s), "probe");
  for (int it = 0; it < 4; ++it) {
    if (it == 3) sqnorm_of(x, BHT_F64, r, acc.as<double>(), s);
    ck(launch_gemm_f64(rows, 1, r, 1.0, X, r, 1, x, 1, 1, 0.0, y.as<double>(), 1, 1, s), "X x");
    ck(cudaMemcpyAsync(z, x, sizeof(double) * r, cudaMemcpyDeviceToDevice, s), "copy");
    ck(launch_gemm_f64(r, 1, rows, 1.0, X, 1, r, y.as<double>(), 1, 1, -1.0, z, 1, 1, s), "X^T y - x");
    std::swap(x, z);
  }
  sqnorm_of(x, BHT_F64, r, acc.as<double>() + 1, s);
  double h[2];
  ck(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H probe");
  ck(cudaStreamSynchronize(s), "sync");
  if (!(h[0] > 0.0)) return h[1] > 0.0 ? 1.0 : 0.0;
  return std::sqrt(h[1] / h[0]);
}

// Estimate of ||V^T X||_2 for V (rows x r0) and X (rows x k) with orthonormal columns: two power steps
// on (V^T X)^T (V^T X) from a pseudo-random start, each four matrix-vector products (the ratio of the
// last two iterates' norms).
double cross_error(const double* V, int64_t r0, const double* X, int64_t k, int64_t rows, cudaStream_t s) {
  if (r0 <= 0 || k <= 0) return 0.0;
  DBuf v(sizeof(double) * (k + r0), s), y(sizeof(double) * rows, s), acc(sizeof(double) * 2, s);
  double* x = v.as<double>();
  double* z = x + k;
  ck(launch_fill_uniform(x, k, 0x63726f7373ull, s), "probe");
  ck(cudaMemsetAsync(acc.p, 0, sizeof(double) * 2, s), "memset");
  for (int it = 0; it < 2; ++it) {
    if (it == 1) sqnorm_of(x, BHT_F64, k, acc.as<double>(), s);
    ck(launch_gemm_f64(rows, 1, k, 1.0, X, k, 1, x, 1, 1, 0.0, y.as<double>(), 1, 1, s), "X x");
    ck(launch_gemm_f64(r0, 1, rows, 1.0, V, 1, r0, y.as<double>(), 1, 1, 0.0, z, 1, 1, s), "V^T y");
    if (it == 1) break;
    ck(launch_gemm_f64(rows, 1, r0, 1.0, V, r0, 1, z, 1, 1, 0.0, y.as<double>(), 1, 1, s), "V z");
    ck(launch_gemm_f64(k, 1, rows, 1.0, X, 1, k, y.as<double>(), 1, 1, 0.0, x, 1, 1, s), "X^T y");
  }
  sqnorm_of(z, BHT_F64, r0, acc.as<double>() + 1, s);
  double h[2];
  ck(cudaMemcpyAsync(h, acc.p, sizeof(h), cudaMemcpyDeviceToHost, s), "D2H probe");
  ck(cudaStreamSynchronize(s), "sync");
  if (!(h[0] > 0.0)) return h[1] > 0.0 ? 1.0 : 0.0;
  return std::sqrt(h[1] / h[0]);
}

// Newton-Schulz steps until the estimated orthonormality error is below 1e-12 (none when the
// columns already are orthonormal to that level; at most max_iters). When steps ran, the result is
// probed again: columns still further than 1e-10 from orthonormal fail with BHT_ENUMERIC, so a basis
// that is not orthonormal never reaches a truncation or a projection.
void orthonormalise(double* X, int64_t rows, int64_t r, cudaStream_t s, int max_iters) {
  const double e0 = orth_error(X, rows, r, s);
  double e = e0;
  int iters = 0;
  while (e > 1e-12 && iters < max_iters) {
    e = 0.75 * e * e + 1e-16;
    ++iters;
  }
  if (iters == 0) return;
  newton_schulz(X, rows, r, s, iters);
  const double e1 = orth_error(X, rows, r, s);
  if (!(e1 <= 1e-10)) {
    char msg[160];
    std::snprintf(msg, sizeof(msg),
                  "a basis of %lld columns is not orthonormal (error %.3g; %.3g before %d Newton-Schulz steps)",
                  (long long)r, e1, e0, iters);
    fail(BHT_ENUMERIC, msg);
  }
}

// Stage 2: orthonormal eigenvectors of the r largest eigenvalues, [n][r] row-major, owned by the caller.
double* eig_vectors64(EigOut& eo, int64_t r, cudaStream_t s) {
  const int64_t n = eo.n;
  double* U = static_cast<double*>(dalloc(sizeof(double) * n * std::max<int64_t>(r, 1), s));
  if (r == 0) return U;
  DBuf scratch(eig_vectors_scratch_bytes(n, r), s);
  ck(launch_eig_vectors(n, r, eo.lam.as<double>(), U, eo.work.p, scratch.p, s), "eigenvectors");
  orthonormalise(U, n, r, s, 3);
  return U;
}

void check_status_word(int* d_status, cudaStream_t s) {
  int h = 0;
  ck(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "status readback");
  ck(cudaStreamSynchronize(s), "sync");
  if (h != 0) {
    cudaMemsetAsync(d_status, 0, sizeof(int), s);
    fail((bht_status)h, "a bounded device-side wait gave up (eigensolver barrier)");
  }
}

void check_status(bht_state* st, cudaStream_t s) { check_status_word(st->d_status, s); }

// Whether every eigenvalue of the n x n Gram matrix G (device) exceeds eps_nw2, certified by a Cholesky
// factorisation of G less a shift that covers its rounding (chol.cu). Then the tail rule of
// eq. ht_leaf_svd keeps all n directions: the energy discarded with n - 1 kept is the smallest
// eigenvalue. No certificate (a pivot <= 0) says nothing either way.
bool certify_full_rank(const double* G, int64_t n, double eps_nw2, int* d_status, cudaStream_t s) {
  DBuf work(spd_test_workspace_bytes(n), s), v(sizeof(int), s);
  ck(launch_spd_test(G, n, eps_nw2, work.p, v.as<int>(), d_status, s), "full-rank certificate");
  check_status_word(d_status, s);
  int h = 0;
  ck(cudaMemcpyAsync(&h, v.p, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H verdict");
  ck(cudaStreamSynchronize(s), "sync");
  return h == 1;
}

int num_sms() {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return std::max(nsm, 1);
}

// Whether the Householder route to the complement of k orthonormal columns in R^c fits: its rows in
// the shared memory of at most one CTA per SM, and, when the reflectors are applied, a row of length c
// per warp plus at least one staged reflector.
bool house_fits(int64_t c, int64_t k) {
  const int64_t nsm = num_sms();
  const int64_t rpb = std::max<int64_t>(8, (c + nsm - 1) / nsm);
  return sizeof(double) * (rpb * k + 2 * k + rpb) <= 200 * 1024 && sizeof(double) * c * 9 <= 200 * 1024;
}

// Which route to the complement of k columns in R^c, applied to a rows, is cheaper. Householder: k
// sequential reflector steps (one grid barrier each, about 5 us) and a (2ck - k^2) FP64 FMAs to
// apply them. Randomized: an eigensolve of size m = c - k + 8 (about 11 us per row of the matrix:
// tridiagonalisation, eigenvalues, eigenvectors, back-transformation) and FP64 GEMMs of about
// 4ckm + 2cm^2 + ac(c - k) FMAs. The FP64 rate assumed is 0.25 FMA per ns (about 40 % of the
// nominal peak, what the library's FP64 kernels reach).
bool house_preferred(int64_t a, int64_t c, int64_t k) {
  if (!house_fits(c, k)) return false;
  const double rate = 0.25e3;  // FMAs per microsecond
  const double m = (double)(c - k + 8);
  const double t_house = 5.0 * (double)k + (double)a * (2.0 * (double)c * (double)k - (double)k * (double)k) / rate;
  const double t_rand = 11.0 * m + (4.0 * (double)c * (double)k * m + 2.0 * (double)c * m * m +
                                    (double)a * (double)c * (double)(c - k)) / rate;
  return t_house <= t_rand;
}

// Orthonormal basis [n][n - r] of the orthogonal complement of the orthonormal columns V [n][r]
// (caller owns it): the last n - r columns of V's Householder QR when that route is the cheaper,
// else a randomized route. X = (I - V V^T) Omega for a deterministic pseudo-random Omega with c + 8 columns
// spans the complement (c = n - r); its orthonormal basis is X Z Lambda^{-1/2} from the c leading
// eigenpairs of X^T X, after which one more pass against V and Newton-Schulz steps restore FP64
// orthogonality. A random start avoids the clusters of tiny eigenvalues that an eigenvector
// route through the discarded part of a Gram spectrum would meet.
double* complement_of(const double* V, int64_t n, int64_t r, uint64_t seed, int* d_status, cudaStream_t s) {
  const int64_t c = n - r;
  double* Q = static_cast<double*>(dalloc(sizeof(double) * (size_t)std::max<int64_t>(n * c, 1), s));
  if (c <= 0) return Q;
  if (r == 0) {
    ck(launch_fill_identity(Q, n, s), "identity");
    return Q;
  }
  if (house_preferred(n, n, r)) {
    try {  // the last n - r columns of the Householder QR of V
      DBuf hw(house_workspace_bytes(n, r, num_sms()), s);
      ck(launch_house_complement(nullptr, n, n, V, r, Q, hw.p, d_status, s), "Householder complement");
      check_status_word(d_status, s);
    } catch (...) {
      dfree(Q, s);
      throw;
    }
    return Q;
  }
  try {
    const int64_t k = std::min<int64_t>(n, c + 8);
    DBuf X(sizeof(double) * n * k, s), W(sizeof(double) * r * std::max(k, c), s);
    ck(launch_fill_uniform(X.as<double>(), n * k, seed, s), "random start");
    ck(launch_gemm_f64(r, k, n, 1.0, V, 1, r, X.as<double>(), k, 1, 0.0, W.as<double>(), k, 1, s), "V^T X");
    ck(launch_gemm_f64(n, k, r, -1.0, V, r, 1, W.as<double>(), k, 1, 1.0, X.as<double>(), k, 1, s), "X -= V W");
    DBuf M(sizeof(double) * k * k, s);
    ck(launch_gemm_f64(k, k, n, 1.0, X.as<double>(), 1, k, X.as<double>(), k, 1, 0.0, M.as<double>(), k, 1, s),
       "X^T X");
    EigOut eo;
    eig_tridiag64(M.as<double>(), k, eo, d_status, s);
    check_status_word(d_status, s);
    ck(launch_eig_bisect(k, eo.work.p, eo.lam.as<double>(), 0, k, s), "eigenvalues");
    eo.computed = k;
    DBuf Z;
    Z.p = eig_vectors64(eo, c, s);
    Z.s = s;
    ck(launch_scale_cols_invsqrt(Z.as<double>(), k, c, eo.lam.as<double>(), s), "Z Lambda^-1/2");
    ck(launch_gemm_f64(n, c, k, 1.0, X.as<double>(), k, 1, Z.as<double>(), c, 1, 0.0, Q, c, 1, s), "X Z");
    ck(launch_gemm_f64(r, c, n, 1.0, V, 1, r, Q, c, 1, 0.0, W.as<double>(), c, 1, s), "V^T Q");
    ck(launch_gemm_f64(n, c, r, -1.0, V, r, 1, W.as<double>(), c, 1, 1.0, Q, c, 1, s), "Q -= V W");
    orthonormalise(Q, n, c, s, 3);
    check_status_word(d_status, s);
  } catch (...) {
    dfree(Q, s);
    throw;
  }
  return Q;
}

uint64_t complement_seed(int id, int64_t n_items) {
  return 0x42485452495345ull ^ ((uint64_t)id << 40) ^ (uint64_t)n_items;
}

// Stage host data to the device when needed.
const void* stage_input(const void* Y, int dtype, int64_t numel, DBuf& staging, cudaStream_t s) {
  if (is_device_ptr(Y)) return Y;
  staging = DBuf(dtype_size(dtype) * (size_t)numel, s);
  ck(cudaMemcpyAsync(staging.p, Y, dtype_size(dtype) * (size_t)numel, cudaMemcpyHostToDevice, s), "H2D batch");
  return staging.p;
}

double sqnorm_of(const void* x, int dtype, int64_t n, double* d_acc, cudaStream_t s) {
  note_read(x);
  ck(cudaMemsetAsync(d_acc, 0, sizeof(double), s), "memset");
  if (dtype == BHT_F32)
    ck(launch_sqnorm<float>(static_cast<const float*>(x), n, d_acc, s), "sqnorm");
  else
    ck(launch_sqnorm<double>(static_cast<const double*>(x), n, d_acc, s), "sqnorm");
  return 0.0;
}

// Step 1 of Algorithm 2: project a batch through every layer with the current cores.
// Mode products on distinct axes commute, so every leaf is contracted first
// (the mixed form always takes the innermost axis and rotates the result to
// the front, which after d steps restores the mode order), then the transfer
// nodes layer by layer. norm_y (nullable): ||Y||^2 when a kernel folded it.
LTensor project_all(const bht_state* st, const void* Y, int dtype, int64_t N, const Arith& ar, cudaStream_t s,
                    double* norm_acc = nullptr, bool* norm_done = nullptr, double* resid = nullptr) {
  const bht_tree& t = st->tree;
  LTensor C = input_tensor(t, Y, dtype, N);
  if (norm_done) *norm_done = false;
  auto qcols = [&](int id) { return st->rows(id) - st->rank[id]; };
  if (ar.mixed) {
    // small leaves two modes at a time from the outermost mode (one read of the batch for the first
    // two); the energy each pass removes, ||in||^2 - ||out||^2, goes to the skip test's sum
    int m0 = 0;
    while (ar.pairs && m0 + 1 < t.d && C.dtype == BHT_F32 && (reinterpret_cast<uintptr_t>(C.ptr) & 15) == 0) {
      if (m0 > 0 && m0 + 3 == t.d) {
        // the last three leaves in one read of the (small) intermediate
        const int id1 = t.leaf_of_mode[m0], id2 = t.leaf_of_mode[m0 + 1], id3 = t.leaf_of_mode[m0 + 2];
        int64_t A = N;
        for (int k = 0; k < m0; ++k) A *= C.dims[k];
        const int64_t n1 = C.dims[m0], n2 = C.dims[m0 + 1], n3 = C.dims[m0 + 2];
        const int64_t r1 = st->rank[id1], r2 = st->rank[id2], r3 = st->rank[id3];
        if (tri_project_supported(A, n1, n2, n3, r1, r2, r3)) {
          LTensor nxt;
          nxt.dtype = BHT_F32;
          nxt.N = C.N;
          nxt.dims = C.dims;
          nxt.node = C.node;
          nxt.dims[m0] = r1;
          nxt.dims[m0 + 1] = r2;
          nxt.dims[m0 + 2] = r3;
          nxt.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(nxt.numel(), 1), s);
          nxt.ptr = nxt.own.p;
          note_read(C.ptr);
          ck(launch_tri_project(static_cast<const float*>(C.ptr), A, (int)n1, (int)n2, (int)n3, st->U[id1], (int)r1,
                                (int)r1, st->U[id2], (int)r2, (int)r2, st->U[id3], (int)r3, (int)r3,
                                nxt.own.as<float>(), nullptr, nullptr, resid, ar.d_status, s),
             "three-mode projection");
          C = std::move(nxt);
          m0 = t.d;
          break;
        }
      }
      const int ida = t.leaf_of_mode[m0], idb = t.leaf_of_mode[m0 + 1];
      int64_t A = N, B = 1;
      for (int k = 0; k < m0; ++k) A *= C.dims[k];
      for (int k = m0 + 2; k < t.d; ++k) B *= C.dims[k];
      const int64_t na = C.dims[m0], nb = C.dims[m0 + 1], ra = st->rank[ida], rb = st->rank[idb];
      if (!pair_project_supported(A, na, nb, B, ra, rb)) break;
      LTensor nxt;
      nxt.dtype = BHT_F32;
      nxt.N = C.N;
      nxt.dims = C.dims;
      nxt.node = C.node;
      nxt.dims[m0] = ra;
      nxt.dims[m0 + 1] = rb;
      nxt.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(nxt.numel(), 1), s);
      nxt.ptr = nxt.own.p;
      note_read(C.ptr);
      ck(launch_pair_project(static_cast<const float*>(C.ptr), A, (int)na, (int)nb, B, st->U[ida], (int)ra, (int)ra,
                             st->U[idb], (int)rb, (int)rb, nxt.own.as<float>(), m0 == 0 ? norm_acc : nullptr, nullptr,
                             resid, ar.d_status, s),
         "two-mode projection");
      if (m0 == 0 && norm_done) *norm_done = norm_acc != nullptr;
      C = std::move(nxt);
      m0 += 2;
    }
    if (m0 == 0) {
      for (int step = 0; step < t.d; ++step) {
        const int ax = (int)C.dims.size() - 1;
        const int id = C.node[ax];
        bool used = false;
        LTensor nxt = ttm_proj_resid(C, ax, st->U[id], st->rank[id], st->Q[id], qcols(id), true, ar, s,
                                     step == 0 && !ar.tight ? norm_acc : nullptr, &used, resid, -1, st);
        if (step == 0 && norm_done) *norm_done = used;
        C = std::move(nxt);
      }
    } else {
      // the remaining leaves one axis at a time, in place
      for (int m = m0; m < t.d; ++m) {
        const int id = t.leaf_of_mode[m];
        LTensor nxt = ttm_proj_resid(C, C.axis_of(id), st->U[id], st->rank[id], st->Q[id], qcols(id), false, ar, s,
                                     nullptr, nullptr, resid, -1, st);
        C = std::move(nxt);
      }
    }
  } else {
    std::vector<int> ids;
    std::vector<const double*> Us;
    std::vector<int64_t> rs;
    for (int m = 0; m < t.d; ++m) {
      const int id = t.leaf_of_mode[m];
      ids.push_back(id);
      Us.push_back(st->U[id]);
      rs.push_back(st->rank[id]);
    }
    C = project_layer(std::move(C), ids, Us, rs, ar, s);
  }
  for (int layer = t.p - 1; layer >= 1; --layer) {
    reshape_to_layer(t, C, layer);
    std::vector<int> ids;
    std::vector<const double*> Us;
    std::vector<int64_t> rs;
    for (int id : t.layers[layer]) {
      if (t.nodes[id].leaf()) continue;  // already contracted
      if (st->ident[id]) continue;       // the identity: nothing to apply, nothing removed
      ids.push_back(id);
      Us.push_back(st->U[id]);
      rs.push_back(st->rank[id]);
    }
    if (ids.empty()) continue;
    // small products in place on the FP32 SIMT kernel (the rule of project_layer)
    const bool small = ar.mixed && small_products(C, rs);
    if (ar.mixed && !ar.tight && !small && resid && C.dtype == BHT_F32) {
      std::vector<const double*> Qs;
      std::vector<int64_t> qcs;
      for (int id : ids) {
        Qs.push_back(st->Q[id]);
        qcs.push_back(qcols(id));
      }
      C = project_layer_tc(std::move(C), ids, Us, rs, &Qs, &qcs, resid, ar, s, st);
    } else if (ar.mixed && !ar.tight && !small && C.dtype == BHT_F32) {
      C = project_layer_tc(std::move(C), ids, Us, rs, nullptr, nullptr, nullptr, ar, s, st);
    } else if (ar.mixed && (resid || small)) {
      std::vector<std::pair<int, int64_t>> ops;
      for (size_t k = 0; k < ids.size(); ++k) ops.push_back({C.axis_of(ids[k]), rs[k]});
      for (int k : best_order(C.dims, ops)) {
        const int id = ids[k];
        LTensor nxt = ttm_proj_resid(C, C.axis_of(id), st->U[id], rs[k], st->Q[id], qcols(id), false, ar, s,
                                     nullptr, nullptr, resid, -1, st);
        C = std::move(nxt);
      }
    } else {
      C = project_layer(std::move(C), ids, Us, rs, ar, s);
    }
  }
  return C;  // [N][r11][r12]
}

// Run work(k, stream_k) for the n nodes of a tree layer at the same time: one host thread and one
// CUDA stream per node, each starting after the work already queued on s; s then waits for all of
// them. The nodes of a layer are independent (their Gram matrices, eigensolves and bases touch only
// their own state), and a node's chain is a sequence of small FP64 kernels separated by host
// decisions, so running the chains side by side fills SMs one chain alone leaves idle. Errors are
// rethrown in the calling thread; launch counts and profiles are added to its counters.
template <typename F>
void run_nodes(int n, cudaStream_t s, F&& work) {
  if (n <= 0) return;
  if (n == 1) {
    work(0, s);
    return;
  }
  int dev = 0;
  ck(cudaGetDevice(&dev), "cudaGetDevice");
  const uint32_t mask = g_prof_mask;
  const void* batch = g_batch;
  cudaEvent_t ready = nullptr;
  ck(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "event");
  ck(cudaEventRecord(ready, s), "event record");
  std::vector<cudaStream_t> ss(n, nullptr);
  std::vector<cudaEvent_t> done(n, nullptr);
  for (int k = 0; k < n; ++k) {
    ck(cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking), "stream");
    ck(cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming), "event");
    ck(cudaStreamWaitEvent(ss[k], ready, 0), "stream wait");
  }
  std::vector<int> err_status(n, BHT_OK);
  std::vector<std::string> err_msg(n);
  std::vector<ThreadCounters> cnt(n);
  std::vector<std::thread> th;
  for (int k = 0; k < n; ++k) {
    th.emplace_back([&, k] {
      cudaSetDevice(dev);
      g_prof_mask = mask;
      g_batch = batch;
      try {
        work(k, ss[k]);
      } catch (const Fail& f) {
        err_status[k] = f.st;
        err_msg[k] = g_err;
      } catch (const std::bad_alloc&) {
        err_status[k] = BHT_ENOMEM;
        err_msg[k] = "host allocation failed";
      } catch (...) {
        err_status[k] = BHT_ECUDA;
        err_msg[k] = "unexpected host exception";
      }
      cudaEventRecord(done[k], ss[k]);
      cnt[k] = take_thread_counters();
      g_batch = nullptr;
    });
  }
  for (auto& t : th) t.join();
  for (int k = 0; k < n; ++k) {
    add_thread_counters(cnt[k]);
    cudaStreamWaitEvent(s, done[k], 0);
    cudaEventDestroy(done[k]);
    cudaStreamDestroy(ss[k]);
  }
  cudaEventDestroy(ready);
  for (int k = 0; k < n; ++k)
    if (err_status[k] != BHT_OK) fail((bht_status)err_status[k], err_msg[k]);
}

// Predictor forward pass on X (device, [B][F] fp32) into out (device, [B][2] fp32). With `keep`
// the intermediates stay in the given buffers for the backward pass.
struct MlpActs {
  DBuf xq, pre1, h1, pre2, h2, out;
};

void mlp_forward(const bht_mlp* net, const float* X, int64_t B, MlpActs& A, cudaStream_t s) {
  const int F = net->f_in, H = net->hidden;
  A.xq = DBuf(sizeof(__nv_bfloat16) * B * F, s);
  A.pre1 = DBuf(sizeof(float) * B * H, s);
  A.h1 = DBuf(sizeof(__nv_bfloat16) * B * H, s);
  A.pre2 = DBuf(sizeof(float) * B * H, s);
  A.h2 = DBuf(sizeof(__nv_bfloat16) * B * H, s);
  A.out = DBuf(sizeof(float) * B * 2, s);
  ck(launch_mlp_round_input(X, B * F, A.xq.as<__nv_bfloat16>(), s), "mlp input");
  ck(launch_mlp_linear(A.xq.as<__nv_bfloat16>(), B, F, net->wq + net->oW1(), net->w + net->ob1(), H,
                       A.pre1.as<float>(), A.h1.as<__nv_bfloat16>(), nullptr, s),
     "mlp layer 1");
  ck(launch_mlp_linear(A.h1.as<__nv_bfloat16>(), B, H, net->wq + net->oW2(), net->w + net->ob2(), H,
                       A.pre2.as<float>(), A.h2.as<__nv_bfloat16>(), nullptr, s),
     "mlp layer 2");
  ck(launch_mlp_linear(A.h2.as<__nv_bfloat16>(), B, H, net->wq + net->oW3(), net->w + net->ob3(), 2, nullptr, nullptr,
                       A.out.as<float>(), s),
     "mlp layer 3");
}

// Truncations (non-root nodes) on the layers 1 .. layer.
int svds_through(const bht_tree& t, int layer) {
  int n = 0;
  for (int l = 1; l <= layer; ++l) n += (int)t.layers[l].size();
  return n;
}

// Projection of a layer's nodes that also adds the energy it removes (on each node's complement) to
// *removed (device double); see ttm_proj_resid.
LTensor project_layer_removed(LTensor C, const std::vector<int>& ids, const std::vector<double*>& U,
                              const std::vector<double*>& Q, const std::vector<int64_t>& rank, const bht_tree& t,
                              const std::vector<int64_t>& rows, const Arith& ar, cudaStream_t s, double* removed) {
  std::vector<std::pair<int, int64_t>> ops;
  for (int id : ids) ops.push_back({C.axis_of(id), rank[id]});
  for (int k : best_order(C.dims, ops)) {
    const int id = ids[k];
    LTensor nxt = ttm_proj_resid(C, C.axis_of(id), U[id], rank[id], Q[id], rows[id] - rank[id], false, ar, s, nullptr,
                                 nullptr, removed);
    C = std::move(nxt);
  }
  (void)t;
  return C;
}

// App. C: the error spent after a layer, eps_l^2, from the FP64 norms (FP64 form) or the energy the
// projections removed (mixed form); the tolerance of the next layer is the rest of the budget spread
// over the truncations still to come.
double adaptive_eps_nw2(double eps_abs2, double spent2, int svd_rem) {
  return std::max(eps_abs2 - std::max(spent2, 0.0), 0.0) / std::max(svd_rem, 1);
}

Arith make_arith(int precision, double eps_rel, int* d_status) {
  Arith ar;
  ar.mixed = precision == BHT_PREC_MIXED;
  ar.tight = eps_rel < 1e-3;
  ar.pairs = ar.mixed && eps_rel >= 5e-3;
  ar.d_status = d_status;
  return ar;
}

// out (device, n elements of `out_dtype`) <- C (device, C.dtype)
void copy_convert(const LTensor& C, void* out, int out_dtype, cudaStream_t s) {
  const int64_t n = C.numel();
  if (C.dtype == out_dtype) {
    ck(cudaMemcpyAsync(out, C.ptr, dtype_size(out_dtype) * n, cudaMemcpyDeviceToDevice, s), "copy");
  } else if (C.dtype == BHT_F32) {
    ck(launch_cast<float, double>(static_cast<const float*>(C.ptr), static_cast<double*>(out), n, s), "cast");
  } else {
    ck(launch_cast<double, float>(static_cast<const double*>(C.ptr), static_cast<float*>(out), n, s), "cast");
  }
}

void validate_opts(const bht_opts* o) {
  if (o && o->precision != BHT_PREC_FP64 && o->precision != BHT_PREC_MIXED)
    fail(BHT_EINVAL, "opts.precision must be BHT_PREC_FP64 or BHT_PREC_MIXED");
  if (o && (o->budget < -1 || o->budget > BHT_BUDGET_ADAPTIVE))
    fail(BHT_EINVAL, "opts.budget must be BHT_BUDGET_UNIFORM, BHT_BUDGET_ADAPTIVE or -1");
}

// Root buffer with room for `cap` items of r11 x r12, old items zero-padded (eq. incremental_zero_padding1).
void grow_root(bht_state* st, int64_t r11_old, int64_t r12_old, int64_t r11, int64_t r12, int64_t need,
               cudaStream_t s) {
  const bool reshape = (r11 != r11_old || r12 != r12_old);
  if (!reshape && need <= st->root_cap) return;
  int64_t cap = std::max<int64_t>(st->root_cap, 16);
  while (cap < need) cap *= 2;
  DBuf nr(sizeof(double) * cap * r11 * r12, s);
  if (st->n_items > 0 && reshape)
    ck(launch_copy_pad3<double, double>(st->root, st->n_items, r11_old, r12_old, nr.as<double>(), st->n_items, r11,
                                        r12, s),
       "root re-layout");
  else if (st->n_items > 0)  // the same layout: one contiguous copy
    ck(cudaMemcpyAsync(nr.p, st->root, sizeof(double) * st->n_items * r11 * r12, cudaMemcpyDeviceToDevice, s),
       "root copy");
  dfree(st->root, s);
  st->root = static_cast<double*>(nr.release());
  st->root_cap = cap;
}

}  // namespace

namespace {
// Root-to-leaves expansion (eq. htucker_reconstruction) of N latent items Z (device, FP64,
// [N][r11][r12]) into out ([N][n_1]..[n_d], element type dtype, host or device).
void decode_latent(const bht_state* st, const double* Z, int64_t count, void* out, int32_t dtype, cudaStream_t s) {
  const bht_tree& t = st->tree;
  const Arith ar = make_arith(st->precision, 1.0, st->d_status);
  LTensor C;
  C.dtype = BHT_F64;
  C.N = count;
  C.dims = {st->r11(), st->r12()};
  C.node = {t.nodes[0].child[0], t.nodes[0].child[1]};
  C.ptr = Z;
  for (int layer = 1; layer <= t.p; ++layer) {
    // expand every node of this layer: axis r -> rows
    std::vector<std::pair<int, int64_t>> ops;
    std::vector<int> ids;
    for (int id : t.layers[layer]) {
      ids.push_back(id);
      ops.push_back({C.axis_of(id), st->rows(id)});
    }
    for (int k : best_order(C.dims, ops)) {
      const int id = ids[k];
      const int ax = C.axis_of(id);
      const int64_t r = st->rank[id], a = st->rows(id);
      LTensor nxt = ttm_any(C, ax, st->U[id], r, 1, a, false, ar, s);
      C = std::move(nxt);
    }
    // split transfer axes into their successors' axes (C-order)
    std::vector<int64_t> dims;
    std::vector<int> node;
    for (size_t i = 0; i < C.node.size(); ++i) {
      const TNode& nd = t.nodes[C.node[i]];
      if (nd.layer == layer && !nd.leaf()) {
        dims.push_back(st->rank[nd.child[0]]);
        dims.push_back(st->rank[nd.child[1]]);
        node.push_back(nd.child[0]);
        node.push_back(nd.child[1]);
      } else {
        dims.push_back(C.dims[i]);
        node.push_back(C.node[i]);
      }
    }
    C.dims = dims;
    C.node = node;
  }
  const int64_t n = C.numel();
  if (is_device_ptr(out)) {
    copy_convert(C, out, dtype, s);
  } else {
    DBuf tmp(dtype_size(dtype) * n, s);
    copy_convert(C, tmp.p, dtype, s);
    ck(cudaMemcpyAsync(out, tmp.p, dtype_size(dtype) * n, cudaMemcpyDeviceToHost, s), "D2H");
  }
  ck(cudaStreamSynchronize(s), "sync");
}
}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
#define BHT_API_BEGIN try {
#define BHT_API_END                                     \
  return BHT_OK;                                        \
  }                                                     \
  catch (const Fail& f) {                               \
    return f.st;                                        \
  }                                                     \
  catch (const std::bad_alloc&) {                       \
    g_err = "host allocation failed";                   \
    return BHT_ENOMEM;                                  \
  }                                                     \
  catch (...) {                                         \
    g_err = "unexpected host exception";                \
    return BHT_ECUDA;                                   \
  }

extern "C" {

const char* bht_last_error(void) { return g_err.c_str(); }

bht_status bht_batch_reads(int64_t* count, int32_t reset) {
  if (!count) return BHT_EINVAL;
  *count = g_batch_reads;
  if (reset) g_batch_reads = 0;
  return BHT_OK;
}
const char* bht_version(void) { return "bht-gb300 0.1 (sm_103a)"; }

bht_status bht_profile_enable(uint32_t class_mask) {
  g_prof_mask = class_mask;
  return BHT_OK;
}

bht_status bht_profile_read(double* ms, int64_t* launches, double* flops, double* bytes, int32_t n,
                            int32_t reset) {
  if (n < K_NUM_CLASSES) return BHT_ECAPACITY;
  prof_resolve();
  for (int i = 0; i < n; ++i) {
    if (i >= K_NUM_CLASSES) {
      if (ms) ms[i] = 0.0;
      if (launches) launches[i] = 0;
      if (flops) flops[i] = 0.0;
      if (bytes) bytes[i] = 0.0;
      continue;
    }
    if (ms) ms[i] = g_prof_ms[i];
    if (launches) launches[i] = g_prof_n[i];
    if (flops) flops[i] = g_prof_flops[i];
    if (bytes) bytes[i] = g_prof_bytes[i];
    if (reset) {
      g_prof_ms[i] = 0.0;
      g_prof_n[i] = 0;
      g_prof_flops[i] = 0.0;
      g_prof_bytes[i] = 0.0;
    }
  }
  return BHT_OK;
}

const char* bht_kernel_class_name(int32_t cls) { return kernel_class_name(cls); }

bht_status bht_launch_count(int64_t* count, int32_t reset) {
  if (!count) return BHT_EINVAL;
  *count = g_launches;
  if (reset) g_launches = 0;
  return BHT_OK;
}

bht_status bht_tree_create_balanced(int32_t d, const int64_t* dims, bht_tree** out) {
  BHT_API_BEGIN
  if (!out || !dims) fail(BHT_EINVAL, "null argument");
  if (d < 2 || d > 16) fail(BHT_EINVAL, "d must be in [2, 16]");
  for (int i = 0; i < d; ++i)
    if (dims[i] < 1 || dims[i] > 4096) fail(BHT_EINVAL, "every mode size must be in [1, 4096]");
  bht_tree* t = new bht_tree();
  build_tree(*t, d, dims);
  *out = t;
  BHT_API_END
}

bht_status bht_tree_destroy(bht_tree* tree) {
  delete tree;
  return BHT_OK;
}

bht_status bht_tree_info(const bht_tree* tree, int32_t* depth, int32_t* num_nodes) {
  if (!tree) return BHT_EINVAL;
  if (depth) *depth = tree->p;
  if (num_nodes) *num_nodes = (int32_t)tree->nodes.size();
  return BHT_OK;
}

namespace {
// Leaves-to-root decomposition (Algorithm 1; for `plain`, the leaves-to-root HT algorithm of Sec. 2.3.1
// with the batch as the last leaf of the tree t over (n_1, .., n_d, N)). Y is item-major [N][n_1..n_d]
// in both cases, so for `plain` the batch is the outermost axis of the single tensor until the first
// reshape moves it behind the others.
bht_state* l2r_build(const bht_tree& t, const void* Y, int dtype, int64_t N, double eps_rel, const bht_opts* opts,
                     cudaStream_t s, bool plain) {
  int64_t total = plain ? 1 : N;
  for (auto v : t.dims) total *= v;
  DBuf staging;
  const void* dY = stage_input(Y, dtype, total, staging, s);
  BatchScope batch_scope(dY);

  bht_state* st = new bht_state();
  st->tree = t;
  st->plain = plain;
  st->precision = opts ? opts->precision : BHT_PREC_FP64;
  st->budget = (opts && opts->budget == BHT_BUDGET_ADAPTIVE) ? BHT_BUDGET_ADAPTIVE : BHT_BUDGET_UNIFORM;
  st->rank.assign(t.nodes.size(), 0);
  st->U.assign(t.nodes.size(), nullptr);
  st->Q.assign(t.nodes.size(), nullptr);
  st->ident.assign(t.nodes.size(), nullptr);
  try {
    ck(cudaMalloc(&st->d_status, sizeof(int)), "cudaMalloc status");
    ck(cudaMemsetAsync(st->d_status, 0, sizeof(int), s), "memset status");
    const Arith ar = make_arith(st->precision, eps_rel, st->d_status);
    const bool adaptive = st->budget == BHT_BUDGET_ADAPTIVE;
    // Adjacent axes (a, a + 1) of a layer's intermediate whose two-mode pass applies: both Gram matrices
    // from one read of the intermediate (at the deepest layer, the batch: ||Y||^2 is then the trace of
    // the first of them), and later both projections from one more read.
    struct LeafPair {
      int ax, ida, idb;
      int64_t A, B;
      DBuf Ga, Gb;
    };
    auto find_pairs = [&](const LTensor& Cl, const std::vector<int>& lids) {
      std::vector<LeafPair> out;
      if (!ar.pairs || plain || adaptive || Cl.dtype != BHT_F32 || (reinterpret_cast<uintptr_t>(Cl.ptr) & 15) != 0)
        return out;
      const int na_ax = (int)Cl.dims.size();
      for (int m = 0; m + 1 < na_ax; ++m) {
        const int ida = Cl.node[m], idb = Cl.node[m + 1];
        if (std::find(lids.begin(), lids.end(), ida) == lids.end() ||
            std::find(lids.begin(), lids.end(), idb) == lids.end())
          continue;
        int64_t A = Cl.N, B = 1;
        for (int k = 0; k < m; ++k) A *= Cl.dims[k];
        for (int k = m + 2; k < na_ax; ++k) B *= Cl.dims[k];
        if (!pair_gram_supported(A, Cl.dims[m], Cl.dims[m + 1], B)) continue;
        const int64_t na = Cl.dims[m], nb = Cl.dims[m + 1];
        LeafPair lp{m, ida, idb, A, B, DBuf(sizeof(double) * na * na, s), DBuf(sizeof(double) * nb * nb, s)};
        ck(cudaMemsetAsync(lp.Ga.p, 0, sizeof(double) * na * na, s), "memset");
        ck(cudaMemsetAsync(lp.Gb.p, 0, sizeof(double) * nb * nb, s), "memset");
        note_read(Cl.ptr);
        // the FP32 SIMT pass: the tensor-core one costs 2.7 times as much on 24 x 24 pairs (an MMA carries
        // 24 useful rows of its 128 and costs as much as a full one)
        ck(launch_pair_gram(static_cast<const float*>(Cl.ptr), A, (int)na, (int)nb, B, lp.Ga.as<double>(),
                            lp.Gb.as<double>(), st->d_status, s, false),
           "two-mode Gram pass");
        out.push_back(std::move(lp));
        ++m;
      }
      return out;
    };
    std::vector<LeafPair> pairs =
        find_pairs(input_tensor(t, dY, dtype, N), std::vector<int>(t.layers[t.p].begin(), t.layers[t.p].end()));
    DBuf acc(sizeof(double) * 2, s);
    ck(cudaMemsetAsync(acc.p, 0, sizeof(double), s), "memset");
    if (!pairs.empty())
      ck(launch_trace(pairs[0].Ga.as<double>(), t.dims[pairs[0].ax], acc.as<double>(), s), "trace");
    else
      sqnorm_of(dY, dtype, total, acc.as<double>(), s);
    double normY2 = 0.0;
    ck(cudaMemcpyAsync(&normY2, acc.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H norm");
    ck(cudaStreamSynchronize(s), "sync");
    check_status(st, s);
    if (!std::isfinite(normY2)) fail(BHT_ENUMERIC, "the batch holds non-finite values");
    // node-wise tolerance eps_nw = eps_rel ||Y|| / sqrt(2d - 2) (Algorithm 1). The plain HT tree has d + 1
    // modes and one SVD fewer: its layer-1 nodes split one matrix, whose left and right truncations at
    // the same rank remove the same energy, hence sqrt(2 (d + 1) - 3) (Theorem ht_nodewise_error).
    double eps_nw2 = eps_rel * eps_rel * normY2 / (plain ? 2.0 * t.d - 3.0 : 2.0 * t.d - 2.0);
    DBuf removed(sizeof(double), s);
    ck(cudaMemsetAsync(removed.p, 0, sizeof(double), s), "memset");

    LTensor C = input_tensor(t, dY, dtype, N);
    if (plain) {  // one tensor [N][n_1..n_d]: the batch leaf carries the outermost axis
      C.N = 1;
      C.dims.assign(1, N);
      C.node.assign(1, t.leaf_of_mode[t.d - 1]);
      for (int m = 0; m + 1 < t.d; ++m) {
        C.dims.push_back(t.dims[m]);
        C.node.push_back(t.leaf_of_mode[m]);
      }
    }
    for (int layer = t.p; layer >= 1; --layer) {
      if (layer < t.p && plain && C.node[0] == t.leaf_of_mode[t.d - 1]) {
        // move the batch axis behind the others, the tree's order: [b][rest] -> [rest][b]
        LTensor T;
        T.dtype = C.dtype;
        T.N = 1;
        T.dims.assign(C.dims.begin() + 1, C.dims.end());
        T.dims.push_back(C.dims[0]);
        T.node.assign(C.node.begin() + 1, C.node.end());
        T.node.push_back(C.node[0]);
        T.own = DBuf(dtype_size(C.dtype) * (size_t)C.numel(), s);
        T.ptr = T.own.p;
        ck(launch_transpose2d(C.ptr, T.own.p, C.dims[0], C.numel() / C.dims[0], (int)dtype_size(C.dtype), s),
           "transpose");
        C = std::move(T);
      }
      if (layer < t.p) reshape_to_layer(t, C, layer);
      const auto& ids = t.layers[layer];
      if (layer < t.p) pairs = find_pairs(C, std::vector<int>(ids.begin(), ids.end()));
      for (int id : ids)
        if (C.dims[C.axis_of(id)] > 4096)
          fail(BHT_ECAPACITY, "a node's unfolding has more than 4096 rows (the eigensolver's limit)");
      // HOSVD of the layer: every node from the same intermediate, the nodes side by side
      run_nodes((int)ids.size(), s, [&](int k, cudaStream_t sk) {
        const int id = ids[k];
        const int ax = C.axis_of(id);
        const int64_t I = C.dims[ax];
        DBuf status(sizeof(int), sk);
        ck(cudaMemsetAsync(status.p, 0, sizeof(int), sk), "memset status");
        Arith ark = ar;
        ark.d_status = status.as<int>();
        EigOut eo;
        {
          DBuf G(sizeof(double) * I * I, sk);
          const DBuf* pg = nullptr;
          for (const LeafPair& lp : pairs) pg = (lp.ida == id) ? &lp.Ga : (lp.idb == id) ? &lp.Gb : pg;
          if (pg)
            ck(cudaMemcpyAsync(G.p, pg->p, sizeof(double) * I * I, cudaMemcpyDeviceToDevice, sk), "pair Gram");
          else
            gram_any(C, ax, G.as<double>(), ark, sk);
          // an interior node that keeps every direction (eq. ht_leaf_svd with r = I) takes the identity
          // as its basis: U U^T = I is all the truncation states, and the layer's products skip the node.
          // Only possible when the unfolding has at least I columns.
          if (!t.nodes[id].leaf() && I >= 2 && C.numel() / I >= I &&
              certify_full_rank(G.as<double>(), I, eps_nw2, status.as<int>(), sk)) {
            double* U = static_cast<double*>(dalloc(sizeof(double) * I * I, sk));
            ck(launch_fill_identity(U, I, sk), "identity basis");
            st->U[id] = U;
            st->rank[id] = I;
            st->Q[id] = complement_of(U, I, I, complement_seed(id, 0), status.as<int>(), sk);  // empty
            st->ident[id] = U;
            return;
          }
          if (ar.mixed && I <= 32) {
            // a small node of the mixed path: FP32 Jacobi vectors, FP64 Ritz values (ritz.cu); the tail rule
            // on the Ritz values bounds the energy that the kept vectors discard, and the other vectors are
            // their orthonormal complement
            DBuf lam(sizeof(double) * I, sk), V(sizeof(double) * I * I, sk);
            ck(launch_small_ritz(G.as<double>(), I, lam.as<double>(), V.as<double>(), sk), "small eigensolve");
            std::vector<double> hl(I);
            ck(cudaMemcpyAsync(hl.data(), lam.p, sizeof(double) * I, cudaMemcpyDeviceToHost, sk), "D2H Ritz values");
            ck(cudaStreamSynchronize(sk), "sync");
            double tr = 0.0;
            for (double v : hl) tr += v;
            const int64_t r = tail_rank(hl.data(), I, tr, eps_nw2, 1, I);  // eq. ht_leaf_svd, r >= 1
            double* U = static_cast<double*>(dalloc(sizeof(double) * I * r, sk));
            ck(launch_copy_cols(V.as<double>(), I, I, r, U, r, sk), "kept vectors");
            double* Qc = static_cast<double*>(dalloc(sizeof(double) * (size_t)std::max<int64_t>(I * (I - r), 1), sk));
            if (r < I) ck(launch_copy_cols(V.as<double>() + r, I, I, I - r, Qc, I - r, sk), "complement");
            st->U[id] = U;
            st->rank[id] = r;
            st->Q[id] = Qc;
            return;
          }
          eig_tridiag64(G.as<double>(), I, eo, status.as<int>(), sk);
          check_status_word(status.as<int>(), sk);
        }
        const int64_t r = eig_rank64(eo, eps_nw2, 1, I, sk);  // eq. ht_leaf_svd, r >= 1
        double* U = eig_vectors64(eo, r, sk);
        st->U[id] = U;
        st->rank[id] = r;
        // kept for HT-RISE: the residual of a later batch lives in span(Q) (eq. compute_residual)
        st->Q[id] = complement_of(U, I, r, complement_seed(id, 0), status.as<int>(), sk);
      });
      std::vector<const double*> Us;
      std::vector<int64_t> rs;
      std::vector<int> pids;  // the nodes whose product changes the intermediate (not the identity)
      for (int id : ids) {
        if (st->ident[id]) continue;
        pids.push_back(id);
        Us.push_back(st->U[id]);
        rs.push_back(st->rank[id]);
      }
      if (adaptive && layer > 1 && ar.mixed) {
        std::vector<int64_t> rows(t.nodes.size(), 0);
        for (int id : ids) rows[id] = st->rows(id);
        C = project_layer_removed(std::move(C), ids, st->U, st->Q, st->rank, t, rows, ar, s, removed.as<double>());
      } else if (pids.empty()) {
        // every node of the layer keeps its whole space: the intermediate is the layer's result
      } else {
        // the pairs two axes at a time (pairs later in the axis order first, so that the views of the
        // earlier ones keep their sizes), then any other node of the layer
        std::vector<int> rest_ids;
        std::vector<const double*> rest_Us;
        std::vector<int64_t> rest_rs;
        if (!pairs.empty()) {
          for (auto it = pairs.rbegin(); it != pairs.rend(); ++it) {
            const int64_t ra = st->rank[it->ida], rb = st->rank[it->idb];
            const int64_t na = C.dims[it->ax], nb = C.dims[it->ax + 1];
            int64_t B = 1;
            for (size_t k = it->ax + 2; k < C.dims.size(); ++k) B *= C.dims[k];
            if (!pair_project_supported(it->A, na, nb, B, ra, rb) || (reinterpret_cast<uintptr_t>(C.ptr) & 15) != 0) {
              rest_ids.push_back(it->ida);
              rest_ids.push_back(it->idb);
              continue;
            }
            LTensor nxt;
            nxt.dtype = BHT_F32;
            nxt.N = C.N;
            nxt.dims = C.dims;
            nxt.node = C.node;
            nxt.dims[it->ax] = ra;
            nxt.dims[it->ax + 1] = rb;
            nxt.own = DBuf(sizeof(float) * (size_t)std::max<int64_t>(nxt.numel(), 1), s);
            nxt.ptr = nxt.own.p;
            note_read(C.ptr);
            ck(launch_pair_project(static_cast<const float*>(C.ptr), it->A, (int)na, (int)nb, B, st->U[it->ida],
                                   (int)ra, (int)ra, st->U[it->idb], (int)rb, (int)rb, nxt.own.as<float>(), nullptr,
                                   nullptr, nullptr, st->d_status, s),
               "two-mode projection");
            C = std::move(nxt);
          }
          for (size_t k = 0; k < ids.size(); ++k) {
            bool paired = false;
            for (const LeafPair& lp : pairs) paired = paired || lp.ida == ids[k] || lp.idb == ids[k];
            if (!paired && !st->ident[ids[k]]) rest_ids.push_back(ids[k]);
          }
          for (int id : rest_ids) {
            rest_Us.push_back(st->U[id]);
            rest_rs.push_back(st->rank[id]);
          }
          if (!rest_ids.empty()) C = project_layer(std::move(C), rest_ids, rest_Us, rest_rs, ar, s);
        } else {
          C = project_layer(std::move(C), pids, Us, rs, ar, s);
        }
      }
      if (adaptive && layer > 1) {
        // App. C: the rest of the budget over the truncations still to come
        double spent2 = 0.0;
        if (ar.mixed) {
          ck(cudaMemcpyAsync(&spent2, removed.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H removed");
          ck(cudaStreamSynchronize(s), "sync");
        } else {
          DBuf c2(sizeof(double), s);
          sqnorm_of(C.ptr, C.dtype, C.numel(), c2.as<double>(), s);
          double h = 0.0;
          ck(cudaMemcpyAsync(&h, c2.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H norm");
          ck(cudaStreamSynchronize(s), "sync");
          spent2 = normY2 - h;
        }
        eps_nw2 = adaptive_eps_nw2(eps_rel * eps_rel * normY2, spent2, svds_through(t, layer - 1));
      }
    }
    // G_0 = reshape(C, [r11, r12, N]) stored item-major (plain: the one root matrix)
    const int64_t items = plain ? 1 : N;
    grow_root(st, st->r11(), st->r12(), st->r11(), st->r12(), items, s);
    copy_convert(C, st->root, BHT_F64, s);
    st->n_items = items;
    ck(cudaStreamSynchronize(s), "sync");
    return st;
  } catch (...) {
    bht_state_destroy(st);
    throw;
  }
}
}  // namespace


bht_status bht_l2r(const bht_tree* tree, const void* Y, int32_t dtype, int64_t N, double eps_rel,
                   const bht_opts* opts, void* stream, bht_state** out) {
  BHT_API_BEGIN
  if (!tree || !Y || !out) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 1) fail(BHT_EINVAL, "N must be >= 1");
  if (!(eps_rel > 0.0) || !std::isfinite(eps_rel)) fail(BHT_EINVAL, "eps_rel must be positive and finite");
  validate_opts(opts);
  *out = l2r_build(*tree, Y, dtype, N, eps_rel, opts, static_cast<cudaStream_t>(stream), false);
  BHT_API_END
}

bht_status ht_l2r(int32_t d, const int64_t* dims, const void* Y, int32_t dtype, int64_t N, double eps_rel,
                  const bht_opts* opts, void* stream, bht_state** out) {
  BHT_API_BEGIN
  if (!dims || !Y || !out) fail(BHT_EINVAL, "null argument");
  if (d < 2 || d > 15) fail(BHT_EINVAL, "d must be in [2, 15]");
  for (int i = 0; i < d; ++i)
    if (dims[i] < 1 || dims[i] > 4096) fail(BHT_EINVAL, "every mode size must be in [1, 4096]");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 1 || N > 4096) fail(BHT_EINVAL, "the batch is a mode of the tree: N must be in [1, 4096]");
  if (!(eps_rel > 0.0) || !std::isfinite(eps_rel)) fail(BHT_EINVAL, "eps_rel must be positive and finite");
  validate_opts(opts);
  if (opts && opts->budget == BHT_BUDGET_ADAPTIVE) fail(BHT_EINVAL, "the plain HT baseline takes the uniform budget");
  std::vector<int64_t> full(dims, dims + d);
  full.push_back(N);
  bht_tree t;
  build_tree(t, d + 1, full.data());
  *out = l2r_build(t, Y, dtype, N, eps_rel, opts, static_cast<cudaStream_t>(stream), true);
  BHT_API_END
}

namespace {
// Step 1 of Algorithm 2 for one batch, enqueued on s: the projection Cbar onto the current cores,
// ||Y||^2 and the projection error of eq. relative_error_threshold (FP64 form: ||Y||^2 - ||C||^2;
// mixed form: the sum of the energies each node's complement removes), copied with the status word of
// the bounded waits into the pinned slot hp, followed by the event ev. Nothing here waits for the GPU.
struct Step1 {
  LTensor Cbar;
  DBuf acc;
  int64_t reads = 0;     // reads of the batch by the enqueued work
  double* hp = nullptr;  // pinned: ||Y||^2, ||C||^2, projection error, status word (int) in slot 3
  cudaEvent_t ev = nullptr;
  Step1() = default;
  Step1(const Step1&) = delete;
  Step1& operator=(const Step1&) = delete;
  ~Step1() {
    if (ev) cudaEventDestroy(ev);
  }
};

double* pinned_slot(bht_state* st, int k) {
  if (!st->pinned) ck(cudaMallocHost(reinterpret_cast<void**>(&st->pinned), sizeof(double) * 8), "pinned slots");
  return st->pinned + 4 * (k & 1);
}

void step1_enqueue(bht_state* st, const void* dY, int32_t dtype, int64_t N, const Arith& ar, cudaStream_t s,
                   double* hp, Step1& o) {
  int64_t item = 1;
  for (auto v : st->tree.dims) item *= v;
  BatchScope scope(dY);
  const int64_t r0 = g_batch_reads;
  o.acc = DBuf(sizeof(double) * 3, s);
  ck(cudaMemsetAsync(o.acc.p, 0, sizeof(double) * 3, s), "memset");
  bool norm_done = false;
  double* resid = ar.mixed ? o.acc.as<double>() + 2 : nullptr;
  o.Cbar = project_all(st, dY, dtype, N, ar, s, o.acc.as<double>(), &norm_done, resid);
  if (!norm_done) sqnorm_of(dY, dtype, N * item, o.acc.as<double>(), s);
  if (!ar.mixed) sqnorm_of(o.Cbar.ptr, o.Cbar.dtype, o.Cbar.numel(), o.acc.as<double>() + 1, s);
  ck(cudaMemcpyAsync(hp, o.acc.p, sizeof(double) * 3, cudaMemcpyDeviceToHost, s), "D2H norms");
  ck(cudaMemcpyAsync(hp + 3, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, s), "status readback");
  ck(cudaEventCreateWithFlags(&o.ev, cudaEventDisableTiming), "event");
  ck(cudaEventRecord(o.ev, s), "event");
  o.hp = hp;
  o.reads = g_batch_reads - r0;
}

// The skip test of Algorithm 2 on an enqueued Step 1 (waits for its event only).
struct Verdict {
  double h[3];
  double eps_proj, eps_des;
  bool skip;
};

Verdict step1_verdict(bht_state* st, Step1& o, double eps_rel, const Arith& ar, cudaStream_t s) {
  ck(cudaEventSynchronize(o.ev), "sync");
  int hstat = 0;
  std::memcpy(&hstat, o.hp + 3, sizeof(int));
  if (hstat != 0) {
    cudaMemsetAsync(st->d_status, 0, sizeof(int), s);
    fail((bht_status)hstat, "a bounded device-side wait gave up");
  }
  Verdict v;
  std::memcpy(v.h, o.hp, sizeof(v.h));
  if (!std::isfinite(v.h[0])) fail(BHT_ENUMERIC, "the batch holds non-finite values");
  v.eps_des = eps_rel * std::sqrt(v.h[0]);
  v.eps_proj = ar.mixed ? std::sqrt(std::max(v.h[2], 0.0))
                        : std::sqrt(std::max(v.h[0] - v.h[1], 0.0));  // eq. relative_error_threshold
  v.skip = v.eps_proj <= v.eps_des;
  return v;
}

// A skipped batch: only the root grows (eq. incremental_root_concatenate), enqueued on s.
void append_root(bht_state* st, const LTensor& Cbar, int64_t N, cudaStream_t s) {
  const int64_t r11 = st->r11(), r12 = st->r12();
  grow_root(st, r11, r12, r11, r12, st->n_items + N, s);
  copy_convert(Cbar, st->root + st->n_items * r11 * r12, BHT_F64, s);
  st->n_items += N;
}

// Steps 2-3 of Algorithm 2 for a batch whose projection error exceeds eps_des: residuals truncated
// node by node, bases expanded, parents zero padded, the batch re-projected; the new cores live in a
// shadow copy until the commit at the end. reads0: reads of the batch before this call.
void update_expand(bht_state* st, const void* dY, int32_t dtype, int64_t N, double eps_rel, const bht_opts* opts,
                   const Arith& ar, const Verdict& v, int64_t reads0, cudaStream_t s, bht_update_info* info) {
  const bht_tree& t = st->tree;
  BatchScope batch_scope(dY);
  const int64_t reads_in = g_batch_reads;
  const double* h = v.h;
  const double eps_des = v.eps_des, eps_proj = v.eps_proj;
  const int64_t r11_old = st->r11(), r12_old = st->r12();
  // Steps 2-3 layer by layer; the new cores live in a shadow copy until commit
  double eps_nw2 = eps_des * eps_des / (2.0 * t.d - 2.0);
  const int budget = (opts && opts->budget >= 0) ? opts->budget : st->budget;
  DBuf removed(sizeof(double), s);
  ck(cudaMemsetAsync(removed.p, 0, sizeof(double), s), "memset");
  const bool want_feat = opts && (opts->predictor || opts->node_features);
  struct {
    int32_t nodes = 0, skipped = 0, fallback = 0, missed = 0;
  } pstat;
  std::vector<int64_t> rank = st->rank;
  std::vector<double*> U = st->U, Q = st->Q;
  std::vector<double*> fresh;  // buffers created by this call
  auto own = [&](double* p) { fresh.push_back(p); return p; };
  try {
    LTensor C = input_tensor(t, dY, dtype, N);
    for (int layer = t.p; layer >= 1; --layer) {
      if (layer < t.p) reshape_to_layer(t, C, layer);
      const auto& ids = t.layers[layer];
      const int nn = (int)ids.size();
      std::vector<int64_t> alpha(nn), rold(nn), qc(nn);
      std::vector<DBuf> Gs(nn), skw(nn), stat(nn);
      DBuf trd(sizeof(double) * nn, s), feats(sizeof(float) * 66 * nn, s);
      ck(cudaMemsetAsync(trd.p, 0, sizeof(double) * nn, s), "memset");
      for (int k = 0; k < nn; ++k) {
        const int ax = C.axis_of(ids[k]);
        alpha[k] = C.dims[ax];
        rold[k] = rank[ids[k]];
        qc[k] = alpha[k] - rold[k];  // <= 0: U spans R^alpha and the residual vanishes
        if (qc[k] > 4096) fail(BHT_ECAPACITY, "a node's residual space exceeds 4096 dimensions (the eigensolver's limit)");
        stat[k] = DBuf(sizeof(int), s);
        ck(cudaMemsetAsync(stat[k].p, 0, sizeof(int), s), "memset status");
        if (qc[k] <= 0) continue;
        Gs[k] = DBuf(sizeof(double) * qc[k] * qc[k], s);
        if (want_feat) skw[k] = DBuf(sketch_workspace_bytes(qc[k], 128), s);
      }
      // phase 1, the nodes side by side: residual Gram matrices, their exact energies and features.
      // Residual R = (I - U U^T) C_(j) (eq. compute_residual). With Q the orthonormal complement of U,
      // I - U U^T = Q Q^T, so R R^T = Q (W W^T) Q^T for W = Q^T C_(j): the nonzero eigenpairs of the
      // residual Gram are those of the qc x qc Gram W W^T, mapped through Q.
      run_nodes(nn, s, [&](int k, cudaStream_t sk) {
        if (qc[k] <= 0) return;
        const int id = ids[k];
        const int ax = C.axis_of(id);
        Arith ark = ar;
        ark.d_status = stat[k].as<int>();
        // W = Q^T C_(j): on the tensor cores (axis moved innermost) except at tight tolerances, where the
        // FP32 products' 2^-24 keep the small residual resolved
        LTensor W = (ar.mixed && !ar.tight && C.dtype == BHT_F32)
                        ? project_layer_tc(C.view_copy(), {id}, {Q[id]}, {qc[k]}, nullptr, nullptr, nullptr, ark, sk)
                        : ttm_any(C, ax, Q[id], 1, qc[k], qc[k], false, ark, sk);
        gram_any(W, W.axis_of(id), Gs[k].as<double>(), ark, sk);
        ck(launch_trace(Gs[k].as<double>(), qc[k], trd.as<double>() + k, sk), "residual energy");
        if (want_feat)
          ck(launch_sketch_features(Gs[k].as<double>(), qc[k], 128, std::sqrt(eps_nw2), trd.as<double>() + k,
                                    complement_seed(id, st->n_items) ^ 0x736b65746368ull, skw[k].p,
                                    feats.as<float>() + 66 * k, sk),
             "sketch features");
      });
      std::vector<double> tr(nn, 0.0);
      ck(cudaMemcpyAsync(tr.data(), trd.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s), "D2H energies");
      // the predictor's view of the layer: a node predicted not to expand skips its eigensolve when the
      // exact check (the residual energy) confirms that the truncation keeps nothing
      std::vector<char> skip_eig(nn, 0), pred_expand(nn, 1);
      if (want_feat) {
        std::vector<float> hf(66 * (size_t)nn);
        ck(cudaMemcpyAsync(hf.data(), feats.p, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost, s), "D2H features");
        std::vector<float> ho(2 * (size_t)nn, 0.f);
        if (opts->predictor) {
          MlpActs A;
          mlp_forward(opts->predictor, feats.as<float>(), nn, A, s);
          ck(cudaMemcpyAsync(ho.data(), A.out.p, sizeof(float) * ho.size(), cudaMemcpyDeviceToHost, s), "D2H preds");
          ck(cudaStreamSynchronize(s), "sync");
        } else {
          ck(cudaStreamSynchronize(s), "sync");
        }
        for (int k = 0; k < nn; ++k) {
          if (qc[k] <= 0) continue;
          if (opts->node_features)
            std::memcpy(opts->node_features + 66 * (size_t)ids[k], hf.data() + 66 * k, sizeof(float) * 66);
          if (!opts->predictor) continue;
          ++pstat.nodes;
          pred_expand[k] = ho[2 * k + 1] > 0.f;
          if (!pred_expand[k]) {
            if (tr[k] <= eps_nw2) {
              skip_eig[k] = 1;
              ++pstat.skipped;
            } else {
              ++pstat.fallback;
            }
          }
        }
      } else {
        ck(cudaStreamSynchronize(s), "sync");
      }
      // the tail rule of eq. svd_on_residual keeps nothing when the whole residual energy is within the
      // node's budget (tail(0) = trace(R R^T) <= eps_nw^2 gives r_R = 0): no eigensolve, with or without
      // a predictor
      for (int k = 0; k < nn; ++k)
        if (qc[k] > 0 && tr[k] <= eps_nw2) skip_eig[k] = 1;
      // phase 2, the nodes side by side: eigensolve, truncation and expansion
      std::mutex own_mu;
      auto own_locked = [&](double* p) {
        std::lock_guard<std::mutex> lock(own_mu);
        fresh.push_back(p);
        return p;
      };
      std::vector<int64_t> rRs(nn, 0);
      run_nodes(nn, s, [&](int k, cudaStream_t sk) {
        const int id = ids[k];
        const int64_t a = alpha[k], r0 = rold[k], c = qc[k];
        if (c <= 0) return;
        int* status = stat[k].as<int>();
        // eq. svd_on_residual: r_R >= 0 with tail <= eps_nw^2, at most alpha - r_old new directions
        EigOut eo;
        int64_t rR = 0;
        if (!skip_eig[k]) {
          eig_tridiag64(Gs[k].as<double>(), c, eo, status, sk);
          check_status_word(status, sk);
          rR = eig_rank64(eo, eps_nw2, 0, c, sk, tr[k]);
        }
        if (skip_eig[k]) check_status_word(status, sk);  // the phase-1 kernels' bounded waits
        rRs[k] = rR;
        if (opts && opts->node_labels) {
          opts->node_labels[2 * (size_t)id] = rR;
          opts->node_labels[2 * (size_t)id + 1] = c;
        }
        if (rR == 0) return;
        DBuf Zk;
        Zk.p = eig_vectors64(eo, rR, sk);  // [c][rR]
        Zk.s = sk;
        DBuf UR(sizeof(double) * a * rR, sk);
        ck(launch_gemm_f64(a, rR, c, 1.0, Q[id], c, 1, Zk.as<double>(), rR, 1, 0.0, UR.as<double>(), rR, 1, sk),
           "U_R = Q Z");
        // the complement shrinks to Q times the complement of Z inside R^c
        double* Qn = own_locked(static_cast<double*>(dalloc(sizeof(double) * (size_t)std::max<int64_t>(a * (c - rR), 1), sk)));
        if (c > rR) {
          if (house_preferred(a, c, rR)) {
            // rR Householder reflectors of Z applied to the rows of Q
            DBuf hw(house_workspace_bytes(c, rR, num_sms()), sk);
            ck(launch_house_complement(Q[id], a, c, Zk.as<double>(), rR, Qn, hw.p, status, sk),
               "Householder complement");
          } else {
            DBuf Yc;
            Yc.p = complement_of(Zk.as<double>(), c, rR, complement_seed(id, st->n_items), status, sk);
            Yc.s = sk;
            ck(launch_gemm_f64(a, c - rR, c, 1.0, Q[id], c, 1, Yc.as<double>(), c - rR, 1, 0.0, Qn, c - rR, 1, sk),
               "Q Y");
          }
        }
        DBuf W(sizeof(double) * r0 * rR + 8, sk);
        // two Gram-Schmidt passes against U_old (U_R is orthogonal to U_old in exact arithmetic, and Q keeps
        // it so to rounding level: the passes run only when a probe finds ||U_old^T U_R|| above 1e-13)
        const bool need_gs = r0 > 0 && cross_error(U[id], r0, UR.as<double>(), rR, a, sk) > 1e-13;
        for (int pass = 0; pass < 2 && need_gs; ++pass) {
          ck(launch_gemm_f64(r0, rR, a, 1.0, U[id], 1, r0, UR.as<double>(), rR, 1, 0.0, W.as<double>(), rR, 1, sk),
             "U^T U_R");
          ck(launch_gemm_f64(a, rR, r0, -1.0, U[id], r0, 1, W.as<double>(), rR, 1, 1.0, UR.as<double>(), rR, 1, sk),
             "U_R -= U W");
        }
        orthonormalise(UR.as<double>(), a, rR, sk, 3);
        // expandCore: U^k = [U^{k-1}, U_R] (eq. concatenating_orthonormal_vectors)
        const int64_t rn = r0 + rR;
        double* Un = own_locked(static_cast<double*>(dalloc(sizeof(double) * a * rn, sk)));
        if (r0 > 0) ck(launch_copy_cols(U[id], r0, a, r0, Un, rn, sk), "expand old");
        ck(launch_copy_cols(UR.as<double>(), rR, a, rR, Un + r0, rn, sk), "expand new");
        check_status_word(status, sk);
        U[id] = Un;
        Q[id] = Qn;
        rank[id] = rn;
      });
      std::vector<int> grown_parents;
      for (int k = 0; k < nn; ++k) {
        if (qc[k] > 0 && opts && opts->predictor && pred_expand[k] && rRs[k] == 0) ++pstat.missed;
        if (rRs[k] == 0) continue;
        const int par = t.nodes[ids[k]].parent;
        if (par > 0 && std::find(grown_parents.begin(), grown_parents.end(), par) == grown_parents.end())
          grown_parents.push_back(par);
      }
      // padWithZeros of every parent whose successor grew (eq. incremental_zero_padding1)
      for (int par : grown_parents) {
        const TNode& pn = t.nodes[par];
        const int c0 = pn.child[0], c1 = pn.child[1];
        // child ranks before this layer's expansion
        int64_t ra0 = rank[c0], rb0 = rank[c1];
        for (size_t k = 0; k < ids.size(); ++k) {
          if (ids[k] == c0) ra0 = rold[k];
          if (ids[k] == c1) rb0 = rold[k];
        }
        const int64_t rp = rank[par], ra = rank[c0], rb = rank[c1];
        double* Pn = own(static_cast<double*>(dalloc(sizeof(double) * ra * rb * rp, s)));
        ck(launch_copy_pad3<double, double>(U[par], ra0, rb0, rp, Pn, ra, rb, rp, s), "pad parent");
        U[par] = Pn;
        // the complement gains a unit vector for each new merged coordinate
        const int64_t q0 = ra0 * rb0 - rp, q1 = ra * rb - rp;
        double* Pq = own(static_cast<double*>(dalloc(sizeof(double) * (size_t)std::max<int64_t>(ra * rb * q1, 1), s)));
        ck(launch_copy_pad3<double, double>(Q[par], ra0, rb0, q0, Pq, ra, rb, q1, s), "pad complement");
        ck(launch_unit_cols(Pq, q1, q0, ra0, rb0, ra, rb, s), "complement of new coordinates");
        Q[par] = Pq;
      }
      // Step 1 revisited: project onto the updated cores of the layer (a basis that is still the
      // identity leaves the intermediate as it is)
      std::vector<int> pids;
      std::vector<const double*> Us;
      std::vector<int64_t> rs;
      for (int id : ids) {
        if (st->ident[id] && U[id] == st->ident[id]) continue;
        pids.push_back(id);
        Us.push_back(U[id]);
        rs.push_back(rank[id]);
      }
      const bool adaptive = budget == BHT_BUDGET_ADAPTIVE && layer > 1;
      if (adaptive && ar.mixed) {
        std::vector<int64_t> rows(t.nodes.size(), 0);
        for (int k = 0; k < nn; ++k) rows[ids[k]] = alpha[k];
        C = project_layer_removed(std::move(C), ids, U, Q, rank, t, rows, ar, s, removed.as<double>());
      } else if (!pids.empty()) {
        C = project_layer(std::move(C), pids, Us, rs, ar, s);
      }
      if (adaptive) {
        // App. C on the update: the error spent by the projection onto the updated cores so far
        double spent2 = 0.0;
        if (ar.mixed) {
          ck(cudaMemcpyAsync(&spent2, removed.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H removed");
          ck(cudaStreamSynchronize(s), "sync");
        } else {
          DBuf c2(sizeof(double), s);
          sqnorm_of(C.ptr, C.dtype, C.numel(), c2.as<double>(), s);
          double hc = 0.0;
          ck(cudaMemcpyAsync(&hc, c2.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H norm");
          ck(cudaStreamSynchronize(s), "sync");
          spent2 = h[0] - hc;
        }
        eps_nw2 = adaptive_eps_nw2(eps_des * eps_des, spent2, svds_through(t, layer - 1));
      }
    }
    // eq. incremental_root_concatenate with the root zero-padded in modes 1, 2
    const int64_t r11 = rank[t.nodes[0].child[0]], r12 = rank[t.nodes[0].child[1]];
    grow_root(st, r11_old, r12_old, r11, r12, st->n_items + N, s);
    copy_convert(C, st->root + st->n_items * r11 * r12, BHT_F64, s);
    ck(cudaStreamSynchronize(s), "sync");
  } catch (...) {
    for (double* p : fresh) dfree(p, s);
    cudaStreamSynchronize(s);
    throw;
  }
  // commit: release the replaced cores and any intermediate core superseded within this call
  for (size_t id = 1; id < U.size(); ++id) {
    if (U[id] != st->U[id]) {
      st->ident[id] = nullptr;
      purge_weights(st, st->U[id], s);
      dfree(st->U[id], s);
    }
    if (Q[id] != st->Q[id]) {
      purge_weights(st, st->Q[id], s);
      dfree(st->Q[id], s);
    }
  }
  for (double* p : fresh)
    if (std::find(U.begin(), U.end(), p) == U.end() && std::find(Q.begin(), Q.end(), p) == Q.end()) dfree(p, s);
  st->U = U;
  st->Q = Q;
  st->rank = rank;
  st->n_items += N;
  ck(cudaStreamSynchronize(s), "sync");
  if (info)
    *info = bht_update_info{0, (int32_t)(reads0 + g_batch_reads - reads_in), eps_proj, eps_des, std::sqrt(h[0]),
                            st->n_items, pstat.nodes, pstat.skipped, pstat.fallback, pstat.missed};
}
}  // namespace

bht_status htrise_update(bht_state* st, const void* Y, int32_t dtype, int64_t N, double eps_rel,
                         const bht_opts* opts, void* stream, bht_update_info* info) {
  BHT_API_BEGIN
  if (!st || !Y) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 1) fail(BHT_EINVAL, "N must be >= 1");
  if (!(eps_rel > 0.0) || !std::isfinite(eps_rel)) fail(BHT_EINVAL, "eps_rel must be positive and finite");
  validate_opts(opts);
  if (st->plain) fail(BHT_EINVAL, "HT-RISE appends items along the root; this state holds a plain HT tensor");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t item = 1;
  for (auto v : st->tree.dims) item *= v;
  DBuf staging;
  const void* dY = stage_input(Y, dtype, N * item, staging, s);
  const Arith ar = make_arith(opts ? opts->precision : st->precision, eps_rel, st->d_status);
  // Step 1: project onto the existing cores; the skip test after one synchronisation
  Step1 o;
  step1_enqueue(st, dY, dtype, N, ar, s, pinned_slot(st, 0), o);
  const Verdict v = step1_verdict(st, o, eps_rel, ar, s);
  if (v.skip) {
    append_root(st, o.Cbar, N, s);
    ck(cudaStreamSynchronize(s), "sync");
    if (info)
      *info = bht_update_info{1, (int32_t)o.reads, v.eps_proj, v.eps_des, std::sqrt(v.h[0]), st->n_items, 0, 0, 0, 0};
    return BHT_OK;
  }
  o.Cbar = LTensor();
  update_expand(st, dY, dtype, N, eps_rel, opts, ar, v, o.reads, s, info);
  BHT_API_END
}

bht_status htrise_update_stream(bht_state* st, const void* Y, int32_t dtype, int64_t N, int64_t count,
                                double eps_rel, const bht_opts* opts, void* stream, bht_update_info* infos,
                                int64_t* done) {
  if (done) *done = 0;
  BHT_API_BEGIN
  if (!st || !Y) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 1) fail(BHT_EINVAL, "N must be >= 1");
  if (count < 0) fail(BHT_EINVAL, "count must be >= 0");
  if (!(eps_rel > 0.0) || !std::isfinite(eps_rel)) fail(BHT_EINVAL, "eps_rel must be positive and finite");
  validate_opts(opts);
  if (st->plain) fail(BHT_EINVAL, "HT-RISE appends items along the root; this state holds a plain HT tensor");
  if (count == 0) return BHT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t item = 1;
  for (auto v : st->tree.dims) item *= v;
  const size_t bytes = dtype_size(dtype) * (size_t)(N * item);
  const char* Yc = static_cast<const char*>(Y);
  const bool host = !is_device_ptr(Y);
  const Arith ar = make_arith(opts ? opts->precision : st->precision, eps_rel, st->d_status);
  // room in the root for every item of the stream at the current ranks, so that the appends of skipped
  // updates copy nothing (an expansion re-lays the root out as in htrise_update)
  grow_root(st, st->r11(), st->r12(), st->r11(), st->r12(), st->n_items + count * N, s);
  // host batches: two device buffers, filled on a copy stream while the previous batch computes
  DBuf buf[2];
  cudaStream_t cs = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  struct Cleanup {
    cudaStream_t* cs;
    cudaEvent_t* ev;
    cudaStream_t s;
    ~Cleanup() {
      if (*cs) {
        cudaStreamSynchronize(*cs);
        cudaStreamDestroy(*cs);
      }
      cudaStreamSynchronize(s);
      for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    }
  };
  cudaEvent_t evs[4] = {nullptr, nullptr, nullptr, nullptr};
  Cleanup cleanup{&cs, evs, s};
  if (host) {
    for (int b = 0; b < 2 && b < count; ++b) buf[b] = DBuf(bytes, s);
    ck(cudaStreamSynchronize(s), "sync");
    ck(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "copy stream");
    for (int i = 0; i < 4; ++i) ck(cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming), "event");
    copied[0] = evs[0];
    copied[1] = evs[1];
    freed[0] = evs[2];
    freed[1] = evs[3];
  }
  // batch k into buffer k mod 2, after `left` (the batch two back is done with that buffer)
  auto h2d = [&](int64_t k, cudaEvent_t left) {
    const int b = (int)(k & 1);
    if (left) ck(cudaStreamWaitEvent(cs, left, 0), "wait");
    ck(cudaMemcpyAsync(buf[b].p, Yc + (size_t)k * bytes, bytes, cudaMemcpyHostToDevice, cs), "H2D batch");
    ck(cudaEventRecord(copied[b], cs), "event");
  };
  auto batch = [&](int64_t k) -> const void* {
    if (!host) return Yc + (size_t)k * bytes;
    ck(cudaStreamWaitEvent(s, copied[k & 1], 0), "wait");
    return buf[k & 1].p;
  };
  if (host) {
    h2d(0, nullptr);
    if (count > 1) h2d(1, nullptr);
  }
  // Step 1 of batch k + 1 is enqueued before the skip test of batch k is read: the cores it projects
  // onto are those batch k leaves whenever batch k is skipped; otherwise it is dropped and redone
  std::unique_ptr<Step1> cur(new Step1), nxt;
  const void* dcur = batch(0);
  step1_enqueue(st, dcur, dtype, N, ar, s, pinned_slot(st, 0), *cur);
  for (int64_t k = 0; k < count; ++k) {
    const void* dnext = nullptr;
    cudaEvent_t left = nullptr;  // the point on s after which batch k no longer reads its input
    if (k + 1 < count) {
      dnext = batch(k + 1);
      nxt.reset(new Step1);
      step1_enqueue(st, dnext, dtype, N, ar, s, pinned_slot(st, k + 1), *nxt);
    }
    const Verdict v = step1_verdict(st, *cur, eps_rel, ar, s);
    if (v.skip) {
      append_root(st, cur->Cbar, N, s);
      if (infos)
        infos[k] = bht_update_info{1, (int32_t)cur->reads, v.eps_proj, v.eps_des, std::sqrt(v.h[0]), st->n_items,
                                   0, 0, 0, 0};
      left = cur->ev;  // a skipped batch read its input in Step 1 only
    } else {
      // the speculative Step 1 of batch k + 1 projected onto cores that are about to change
      if (nxt) {
        ck(cudaEventSynchronize(nxt->ev), "sync");
        nxt.reset();
      }
      cur->Cbar = LTensor();
      update_expand(st, dcur, dtype, N, eps_rel, opts, ar, v, cur->reads, s, infos ? infos + k : nullptr);
      if (host) {
        ck(cudaEventRecord(freed[k & 1], s), "event");
        left = freed[k & 1];
      }
      if (k + 1 < count) {
        nxt.reset(new Step1);
        step1_enqueue(st, dnext, dtype, N, ar, s, pinned_slot(st, k + 1), *nxt);
      }
    }
    if (done) *done = k + 1;
    if (host && k + 2 < count) h2d(k + 2, left);
    cur = std::move(nxt);
    dcur = dnext;
  }
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status ht_reconstruct(const bht_state* st, int64_t first, int64_t count, void* out, int32_t dtype,
                          void* stream) {
  BHT_API_BEGIN
  if (!st || !out) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (first < 0 || count < 0 || first + count > st->n_items) fail(BHT_EINVAL, "item range outside the accumulation");
  if (count == 0) return BHT_OK;
  decode_latent(st, st->root + first * st->r11() * st->r12(), count, out, dtype, static_cast<cudaStream_t>(stream));
  BHT_API_END
}

bht_status ht_decode(const bht_state* st, const double* latent, int64_t N, void* out, int32_t dtype, void* stream) {
  BHT_API_BEGIN
  if (!st || (N > 0 && (!latent || !out))) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 0) fail(BHT_EINVAL, "N must be >= 0");
  if (N == 0) return BHT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf staging;
  const double* dZ = static_cast<const double*>(stage_input(latent, BHT_F64, N * st->r11() * st->r12(), staging, s));
  decode_latent(st, dZ, N, out, dtype, s);
  BHT_API_END
}

bht_status ht_relative_test_error(const bht_state* st, const void* X, int32_t dtype, int64_t N, double* rte,
                                  double* item_err, void* stream) {
  BHT_API_BEGIN
  if (!st || !X || !rte) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 1) fail(BHT_EINVAL, "N must be >= 1");
  if (st->plain) fail(BHT_EINVAL, "a plain HT state has no item axis to encode along");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t item = 1;
  for (auto v : st->tree.dims) item *= v;
  DBuf staging;
  const char* dX = static_cast<const char*>(stage_input(X, dtype, N * item, staging, s));
  const Arith ar = make_arith(st->precision, 1.0, st->d_status);
  DBuf acc(sizeof(double) * 2 * N, s);
  ck(cudaMemsetAsync(acc.p, 0, sizeof(double) * 2 * N, s), "memset");
  double* err2 = acc.as<double>();
  double* nrm2 = err2 + N;
  // items in chunks of at most 2^27 decoded FP64 elements (1 GiB)
  const int64_t per = std::max<int64_t>(1, ((int64_t)1 << 27) / item);
  for (int64_t first = 0; first < N; first += per) {
    const int64_t n = std::min(per, N - first);
    const void* xc = dX + dtype_size(dtype) * (size_t)(first * item);
    LTensor C = project_all(st, xc, dtype, n, ar, s);           // encode (Step 1 of Algorithm 2)
    DBuf Z(sizeof(double) * (size_t)C.numel(), s);
    copy_convert(C, Z.p, BHT_F64, s);
    DBuf Xh(sizeof(double) * (size_t)(n * item), s);
    decode_latent(st, Z.as<double>(), n, Xh.p, BHT_F64, s);   // decode (eq. htucker_reconstruction)
    ck(launch_item_errors(xc, dtype, Xh.as<double>(), n, item, err2 + first, nrm2 + first, s), "item errors");
  }
  std::vector<double> h(2 * N);
  ck(cudaMemcpyAsync(h.data(), acc.p, sizeof(double) * 2 * N, cudaMemcpyDeviceToHost, s), "D2H errors");
  ck(cudaStreamSynchronize(s), "sync");
  // eq. generalization_performance: the mean over items of ||X_i - X~_i|| / ||X_i|| (a zero item that
  // decodes to zero has error 0)
  double sum = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double e = h[i] > 0.0 ? std::sqrt(h[i] / h[N + i]) : 0.0;
    if (item_err) item_err[i] = e;
    sum += e;
  }
  *rte = sum / (double)N;
  BHT_API_END
}

bht_status bht_normalize(void* Y, int32_t dtype, int64_t groups, int64_t group_size, int32_t kind, double* params,
                         void* stream) {
  BHT_API_BEGIN
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (kind < BHT_NORM_NONE || kind > BHT_NORM_ZSCORE) fail(BHT_EINVAL, "unknown normalisation");
  if (groups < 0 || group_size < 0) fail(BHT_EINVAL, "negative size");
  if (groups == 0 || group_size == 0) return BHT_OK;
  if (!Y || !params) fail(BHT_EINVAL, "null argument");
  if (!is_device_ptr(Y)) fail(BHT_EINVAL, "Y must be device memory (normalised in place)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool dev = is_device_ptr(params);
  DBuf tmp;
  double* dp = params;
  if (!dev) {
    tmp = DBuf(sizeof(double) * 2 * groups, s);
    dp = tmp.as<double>();
  }
  ck(launch_normalize(Y, dtype, groups, group_size, kind, dp, s), "normalise");
  if (!dev) ck(cudaMemcpyAsync(params, dp, sizeof(double) * 2 * groups, cudaMemcpyDeviceToHost, s), "D2H params");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_denormalize(void* Y, int32_t dtype, int64_t groups, int64_t group_size, const double* params,
                           void* stream) {
  BHT_API_BEGIN
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (groups < 0 || group_size < 0) fail(BHT_EINVAL, "negative size");
  if (groups == 0 || group_size == 0) return BHT_OK;
  if (!Y || !params) fail(BHT_EINVAL, "null argument");
  if (!is_device_ptr(Y)) fail(BHT_EINVAL, "Y must be device memory (restored in place)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf staging;
  const double* dp = static_cast<const double*>(stage_input(params, BHT_F64, 2 * groups, staging, s));
  ck(launch_denormalize(Y, dtype, groups, group_size, dp, s), "denormalise");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_permute_items(const void* Y, int32_t dtype, int64_t N, int32_t d, const int64_t* dims,
                             const int32_t* perm, void* out, void* stream) {
  BHT_API_BEGIN
  if (!Y || !dims || !perm || !out) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (d < 1 || d > 16) fail(BHT_EINVAL, "d must be in [1, 16]");
  if (N < 0) fail(BHT_EINVAL, "N must be >= 0");
  std::vector<int> seen(d, 0), pm(d);
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1) fail(BHT_EINVAL, "every mode size must be >= 1");
    if (perm[k] < 0 || perm[k] >= d || seen[perm[k]]++) fail(BHT_EINVAL, "perm is not a permutation of 0 .. d-1");
    pm[k] = perm[k];
  }
  if (!is_device_ptr(Y) || !is_device_ptr(out)) fail(BHT_EINVAL, "Y and out must be device memory");
  if (Y == out) fail(BHT_EINVAL, "the permutation is out of place");
  if (N == 0) return BHT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ck(launch_permute_items(Y, dtype, N, d, dims, pm.data(), out, s), "permute");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status ht_encode(const bht_state* st, const void* Y, int32_t dtype, int64_t N, double* out, void* stream) {
  BHT_API_BEGIN
  if (!st || (N > 0 && (!Y || !out))) fail(BHT_EINVAL, "null argument");
  if (dtype != BHT_F32 && dtype != BHT_F64) fail(BHT_EINVAL, "dtype must be BHT_F32 or BHT_F64");
  if (N < 0) fail(BHT_EINVAL, "N must be >= 0");
  if (st->plain) fail(BHT_EINVAL, "a plain HT state has no item axis to encode along");
  if (N == 0) return BHT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t item = 1;
  for (auto v : st->tree.dims) item *= v;
  DBuf staging;
  const void* dY = stage_input(Y, dtype, N * item, staging, s);
  const Arith ar = make_arith(st->precision, 1.0, st->d_status);
  LTensor C = project_all(st, dY, dtype, N, ar, s);
  if (is_device_ptr(out)) {
    copy_convert(C, out, BHT_F64, s);
  } else {
    DBuf tmp(sizeof(double) * C.numel(), s);
    copy_convert(C, tmp.p, BHT_F64, s);
    ck(cudaMemcpyAsync(out, tmp.p, sizeof(double) * C.numel(), cudaMemcpyDeviceToHost, s), "copy out");
  }
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_pair_gram(const float* X, int64_t A, int64_t na, int64_t nb, int64_t B, double* Ga, double* Gb,
                         int32_t tensor_cores, void* stream) {
  BHT_API_BEGIN
  if (!X || !Ga || !Gb) fail(BHT_EINVAL, "null argument");
  if (!pair_gram_supported(A, na, nb, B)) fail(BHT_EUNSUPPORTED, "shape outside the two-mode Gram pass");
  if (!is_device_ptr(X) || !is_device_ptr(Ga) || !is_device_ptr(Gb)) fail(BHT_EINVAL, "device pointers required");
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) fail(BHT_EINVAL, "X must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  ck(cudaMemsetAsync(Ga, 0, sizeof(double) * na * na, s), "memset");
  ck(cudaMemsetAsync(Gb, 0, sizeof(double) * nb * nb, s), "memset");
  ck(launch_pair_gram(X, A, (int)na, (int)nb, B, Ga, Gb, status.as<int>(), s, tensor_cores != 0),
     "two-mode Gram pass");
  check_status_word(status.as<int>(), s);
  BHT_API_END
}

bht_status bht_pair_project(const float* X, int64_t A, int64_t na, int64_t nb, int64_t B, const double* Ua,
                            int64_t ra, const double* Ub, int64_t rb, float* out, double* norms, void* stream) {
  BHT_API_BEGIN
  if (!X || !Ua || !Ub || !out) fail(BHT_EINVAL, "null argument");
  if (!pair_project_supported(A, na, nb, B, ra, rb)) fail(BHT_EUNSUPPORTED, "shape outside the two-mode projection");
  if (!is_device_ptr(X) || !is_device_ptr(Ua) || !is_device_ptr(Ub) || !is_device_ptr(out) ||
      (norms && !is_device_ptr(norms)))
    fail(BHT_EINVAL, "device pointers required");
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) fail(BHT_EINVAL, "X must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  ck(launch_pair_project(X, A, (int)na, (int)nb, B, Ua, (int)ra, (int)ra, Ub, (int)rb, (int)rb, out,
                         norms, norms ? norms + 1 : nullptr, norms ? norms + 2 : nullptr, status.as<int>(), s),
     "two-mode projection");
  check_status_word(status.as<int>(), s);
  BHT_API_END
}

bht_status bht_tri_project(const float* X, int64_t A, int64_t n1, int64_t n2, int64_t n3, const double* U1,
                           int64_t r1, const double* U2, int64_t r2, const double* U3, int64_t r3, float* out,
                           double* norms, void* stream) {
  BHT_API_BEGIN
  if (!X || !U1 || !U2 || !U3 || !out) fail(BHT_EINVAL, "null argument");
  if (!tri_project_supported(A, n1, n2, n3, r1, r2, r3)) fail(BHT_EUNSUPPORTED, "shape outside the three-mode projection");
  if (!is_device_ptr(X) || !is_device_ptr(U1) || !is_device_ptr(U2) || !is_device_ptr(U3) || !is_device_ptr(out) ||
      (norms && !is_device_ptr(norms)))
    fail(BHT_EINVAL, "device pointers required");
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) fail(BHT_EINVAL, "X must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  ck(launch_tri_project(X, A, (int)n1, (int)n2, (int)n3, U1, (int)r1, (int)r1, U2, (int)r2, (int)r2, U3, (int)r3,
                        (int)r3, out, norms, norms ? norms + 1 : nullptr, norms ? norms + 2 : nullptr,
                        status.as<int>(), s),
     "three-mode projection");
  check_status_word(status.as<int>(), s);
  BHT_API_END
}

bht_status bht_mode_product(const float* X, int64_t rows, int64_t K, const double* U, int64_t S, int32_t precision,
                            float* out, int64_t R2, double* norms, void* stream) {
  BHT_API_BEGIN
  if (!X || !U || !out) fail(BHT_EINVAL, "null argument");
  if (rows < 1 || K < 1 || S < 1 || R2 < 1 || rows % R2 != 0) fail(BHT_EINVAL, "bad sizes (rows must be a multiple of R2)");
  if (!is_device_ptr(X) || !is_device_ptr(U) || !is_device_ptr(out) || (norms && !is_device_ptr(norms)))
    fail(BHT_EINVAL, "bht_mode_product takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  if (precision == BHT_PREC_MIXED) {
    if (!ttm_tc_supported(K, S, 2)) fail(BHT_EUNSUPPORTED, "shape outside the tensor-core kernel (K % 4 == 0)");
    DBuf W(ttm_tc_weights_bytes(K, S), s);
    ck(launch_prep_tc_weights(U, K, S, S, true, W.as<float>(), 2, s), "weights");
    ck(launch_ttm_tc(X, rows, K, W.as<float>(), S, 2, out, R2, norms, norms ? norms + 1 : nullptr,
                     status.as<int>(), s),
       "tensor-core mode product");
  } else if (precision == BHT_PREC_FP64) {
    // out[(o S + s) R2 + i]: as a TTM over the view [rows / R2][R2][K] it is a transpose; do it per layout
    if (R2 != 1) fail(BHT_EUNSUPPORTED, "the FP64 form writes the new axis innermost (R2 = 1)");
    ck(launch_ttm_f64<float, float>(X, out, U, 1, S, rows, K, 1, S, s), "mode product");
  } else {
    fail(BHT_EINVAL, "precision must be BHT_PREC_FP64 or BHT_PREC_MIXED");
  }
  int h = 0;
  ck(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
  ck(cudaStreamSynchronize(s), "sync");
  if (h) fail((bht_status)h, "a bounded device-side wait gave up (tensor-core pipeline)");
  BHT_API_END
}

bht_status bht_sym_eig(double* G, int64_t n, double* lam, double* U, int64_t r, void* stream) {
  BHT_API_BEGIN
  if (!G || !lam || (r > 0 && !U)) fail(BHT_EINVAL, "null argument");
  if (n < 1 || r < 0 || r > n) fail(BHT_EINVAL, "need 1 <= n and 0 <= r <= n");
  if (n > 4096) fail(BHT_ECAPACITY, "n > 4096");
  if (!is_device_ptr(G) || !is_device_ptr(lam) || (r > 0 && !is_device_ptr(U)))
    fail(BHT_EINVAL, "bht_sym_eig takes device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  EigOut eo;
  eig_values64(G, n, eo, status.as<int>(), s);
  check_status_word(status.as<int>(), s);  // a tridiagonalisation that gave up leaves no valid T
  ck(cudaMemcpyAsync(lam, eo.lam.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s), "copy");
  if (r > 0) {
    DBuf Ur;
    Ur.p = eig_vectors64(eo, r, s);
    Ur.s = s;
    ck(cudaMemcpyAsync(U, Ur.p, sizeof(double) * n * r, cudaMemcpyDeviceToDevice, s), "copy");
  }
  int h = 0;
  ck(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, s), "status");
  ck(cudaStreamSynchronize(s), "sync");
  if (h) fail((bht_status)h, "a bounded device-side wait gave up (eigensolver)");
  BHT_API_END
}

bht_status bht_sym_eig_small(const double* G, int64_t n, double* lam, double* V, void* stream) {
  BHT_API_BEGIN
  if (!G || !lam || !V) fail(BHT_EINVAL, "null argument");
  if (n < 1 || n > 32) fail(BHT_EINVAL, "need 1 <= n <= 32");
  if (!is_device_ptr(G) || !is_device_ptr(lam) || !is_device_ptr(V)) fail(BHT_EINVAL, "device pointers required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ck(launch_small_ritz(G, n, lam, V, s), "small eigensolve");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_eig_min_above(const double* G, int64_t n, double tau, int32_t* above, void* stream) {
  BHT_API_BEGIN
  if (!G || !above) fail(BHT_EINVAL, "null argument");
  if (n < 1) fail(BHT_EINVAL, "need n >= 1");
  if (n > 4096) fail(BHT_ECAPACITY, "n > 4096");
  if (!(tau >= 0.0) || !std::isfinite(tau)) fail(BHT_EINVAL, "tau must be finite and >= 0");
  if (!is_device_ptr(G)) fail(BHT_EINVAL, "bht_eig_min_above takes a device matrix");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf status(sizeof(int), s);
  ck(cudaMemsetAsync(status.p, 0, sizeof(int), s), "memset");
  *above = certify_full_rank(G, n, tau, status.as<int>(), s) ? 1 : 0;
  BHT_API_END
}

bht_status bht_mlp_create(int32_t f_in, int32_t hidden, const float* params, bht_mlp** out) {
  BHT_API_BEGIN
  if (!params || !out) fail(BHT_EINVAL, "null argument");
  if (f_in < 1 || f_in > 4096 || hidden < 1 || hidden > 4096) fail(BHT_EINVAL, "f_in and hidden must be in [1, 4096]");
  bht_mlp* net = new bht_mlp();
  net->f_in = f_in;
  net->hidden = hidden;
  net->P = (int64_t)hidden * f_in + hidden + (int64_t)hidden * hidden + hidden + 2 * (int64_t)hidden + 2;
  const size_t fb = sizeof(float) * (size_t)net->P;
  cudaError_t e = cudaMalloc(&net->w, fb);
  if (e == cudaSuccess) e = cudaMalloc(&net->m, fb);
  if (e == cudaSuccess) e = cudaMalloc(&net->v, fb);
  if (e == cudaSuccess) e = cudaMalloc(&net->g, fb);
  if (e == cudaSuccess) e = cudaMalloc(&net->wq, sizeof(__nv_bfloat16) * (size_t)net->P);
  if (e == cudaSuccess) e = cudaMemcpy(net->w, params, fb, is_device_ptr(params) ? cudaMemcpyDeviceToDevice
                                                                                  : cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->m, 0, fb);
  if (e == cudaSuccess) e = cudaMemset(net->v, 0, fb);
  if (e == cudaSuccess) e = cudaMemset(net->g, 0, fb);
  if (e == cudaSuccess) e = launch_mlp_to_bf16(net->w, net->P, net->wq, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    bht_mlp_destroy(net);
    fail(BHT_ECUDA, cudaGetErrorString(e));
  }
  *out = net;
  BHT_API_END
}

bht_status bht_mlp_destroy(bht_mlp* net) {
  if (!net) return BHT_OK;
  cudaFree(net->w);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->g);
  cudaFree(net->wq);
  delete net;
  return BHT_OK;
}

bht_status bht_mlp_num_params(const bht_mlp* net, int64_t* n) {
  if (!net || !n) return BHT_EINVAL;
  *n = net->P;
  return BHT_OK;
}

bht_status bht_mlp_get_params(const bht_mlp* net, float* out, int64_t cap, float* grad_out) {
  BHT_API_BEGIN
  if (!net || !out) fail(BHT_EINVAL, "null argument");
  if (cap < net->P) fail(BHT_ECAPACITY, "cap < number of parameters");
  ck(cudaMemcpy(out, net->w, sizeof(float) * net->P, cudaMemcpyDefault), "copy parameters");
  if (grad_out) ck(cudaMemcpy(grad_out, net->g, sizeof(float) * net->P, cudaMemcpyDefault), "copy gradient");
  BHT_API_END
}

bht_status bht_mlp_forward(const bht_mlp* net, const float* X, int64_t B, float* out, void* stream) {
  BHT_API_BEGIN
  if (!net || !X || !out) fail(BHT_EINVAL, "null argument");
  if (B < 1) fail(BHT_EINVAL, "B must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf staging;
  const float* dX = static_cast<const float*>(stage_input(X, BHT_F32, B * net->f_in, staging, s));
  MlpActs A;
  mlp_forward(net, dX, B, A, s);
  ck(cudaMemcpyAsync(out, A.out.p, sizeof(float) * 2 * B, cudaMemcpyDefault, s), "copy out");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_mlp_loss_grad(bht_mlp* net, const float* X, const float* T, int64_t B, double* loss, void* stream) {
  BHT_API_BEGIN
  if (!net || !X || !T) fail(BHT_EINVAL, "null argument");
  if (B < 1) fail(BHT_EINVAL, "B must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int F = net->f_in, H = net->hidden;
  DBuf sx, st;
  const float* dX = static_cast<const float*>(stage_input(X, BHT_F32, B * F, sx, s));
  const float* dT = static_cast<const float*>(stage_input(T, BHT_F32, B * 2, st, s));
  MlpActs A;
  mlp_forward(net, dX, B, A, s);
  DBuf dO(sizeof(float) * B * 2, s), da2(sizeof(float) * B * H, s), da1(sizeof(float) * B * H, s);
  DBuf L(sizeof(double), s);
  ck(cudaMemsetAsync(L.p, 0, sizeof(double), s), "memset");
  ck(launch_mlp_loss(A.out.as<float>(), dT, B, dO.as<float>(), L.as<double>(), s), "mlp loss");
  ck(launch_mlp_outer(dO.as<float>(), B, 2, A.h2.as<__nv_bfloat16>(), H, net->g + net->oW3(), net->g + net->ob3(), s),
     "dW3");
  ck(launch_mlp_backprop(dO.as<float>(), B, 2, net->wq + net->oW3(), H, A.pre2.as<float>(), da2.as<float>(), s),
     "da2");
  ck(launch_mlp_outer(da2.as<float>(), B, H, A.h1.as<__nv_bfloat16>(), H, net->g + net->oW2(), net->g + net->ob2(), s),
     "dW2");
  ck(launch_mlp_backprop(da2.as<float>(), B, H, net->wq + net->oW2(), H, A.pre1.as<float>(), da1.as<float>(), s),
     "da1");
  ck(launch_mlp_outer(da1.as<float>(), B, H, A.xq.as<__nv_bfloat16>(), F, net->g + net->oW1(), net->g + net->ob1(), s),
     "dW1");
  double h = 0.0;
  ck(cudaMemcpyAsync(&h, L.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H loss");
  ck(cudaStreamSynchronize(s), "sync");
  if (loss) *loss = h;
  BHT_API_END
}

bht_status bht_mlp_adam_step(bht_mlp* net, double lr, void* stream) {
  BHT_API_BEGIN
  if (!net) fail(BHT_EINVAL, "null argument");
  if (!(lr > 0.0) || !std::isfinite(lr)) fail(BHT_EINVAL, "lr must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  net->steps += 1;
  const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)net->steps));
  const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)net->steps));
  ck(launch_mlp_adam(net->w, net->m, net->v, net->g, net->P, (float)lr, (float)c1, (float)c2, s), "adam");
  ck(launch_mlp_to_bf16(net->w, net->P, net->wq, s), "bf16 copy");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_sketch_features(const double* G, int64_t c, double tol, double norm, uint64_t seed, float* feat,
                               void* stream) {
  BHT_API_BEGIN
  if (!G || !feat) fail(BHT_EINVAL, "null argument");
  if (c < 1 || c > 4096) fail(BHT_EINVAL, "c must be in [1, 4096]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBuf sg;
  const double* dG = static_cast<const double*>(stage_input(G, BHT_F64, c * c, sg, s));
  DBuf work(sketch_workspace_bytes(c, 128), s), f(sizeof(float) * 66, s), n2(sizeof(double), s);
  const double norm2 = norm * norm;
  ck(cudaMemcpyAsync(n2.p, &norm2, sizeof(double), cudaMemcpyHostToDevice, s), "H2D norm");
  ck(launch_sketch_features(dG, c, 128, tol, n2.as<double>(), seed, work.p, f.as<float>(), s), "sketch features");
  ck(cudaMemcpyAsync(feat, f.p, sizeof(float) * 66, cudaMemcpyDefault, s), "copy features");
  ck(cudaStreamSynchronize(s), "sync");
  BHT_API_END
}

bht_status bht_get_ranks(const bht_state* st, int64_t* ranks, int64_t cap) {
  if (!st || !ranks) return BHT_EINVAL;
  const int64_t nn = (int64_t)st->tree.nodes.size();
  if (cap < nn) return BHT_ECAPACITY;
  ranks[0] = st->n_items;
  for (int64_t i = 1; i < nn; ++i) ranks[i] = st->rank[i];
  return BHT_OK;
}

bht_status bht_get_dims(const bht_state* st, int32_t* d, int64_t* dims, int64_t cap) {
  if (!st) return BHT_EINVAL;
  if (d) *d = st->tree.d;
  if (dims) {
    if (cap < st->tree.d) return BHT_ECAPACITY;
    for (int i = 0; i < st->tree.d; ++i) dims[i] = st->tree.dims[i];
  }
  return BHT_OK;
}

bht_status bht_get_core(const bht_state* st, int32_t node, double* host_out, int64_t cap, int64_t* numel) {
  BHT_API_BEGIN
  if (!st) fail(BHT_EINVAL, "null state");
  if (node < 1 || node >= (int32_t)st->tree.nodes.size()) fail(BHT_EINVAL, "node must be in [1, 2d-2]");
  const int64_t n = st->rows(node) * st->rank[node];
  if (numel) *numel = n;
  if (host_out) {
    if (cap < n) fail(BHT_ECAPACITY, "output too small");
    ck(cudaMemcpy(host_out, st->U[node], sizeof(double) * n, cudaMemcpyDeviceToHost), "D2H core");
  }
  BHT_API_END
}

bht_status bht_get_root(const bht_state* st, int64_t first, int64_t count, double* host_out, int64_t cap) {
  BHT_API_BEGIN
  if (!st || !host_out) fail(BHT_EINVAL, "null argument");
  if (first < 0 || count < 0 || first + count > st->n_items) fail(BHT_EINVAL, "item range outside the accumulation");
  const int64_t per = st->r11() * st->r12();
  if (cap < per * count) fail(BHT_ECAPACITY, "output too small");
  if (count)
    ck(cudaMemcpy(host_out, st->root + first * per, sizeof(double) * per * count, cudaMemcpyDeviceToHost),
       "D2H root");
  BHT_API_END
}

bht_status bht_num_elements(const bht_state* st, int64_t* cores_total) {
  if (!st || !cores_total) return BHT_EINVAL;
  int64_t n = 0;
  for (size_t id = 1; id < st->tree.nodes.size(); ++id) n += st->rows((int)id) * st->rank[id];
  n += st->n_items * st->r11() * st->r12();
  *cores_total = n;
  return BHT_OK;
}

bht_status bht_state_destroy(bht_state* st) {
  if (!st) return BHT_OK;
  cudaDeviceSynchronize();
  for (double* p : st->U)
    if (p) cudaFreeAsync(p, nullptr);
  for (double* p : st->Q)
    if (p) cudaFreeAsync(p, nullptr);
  if (st->root) cudaFreeAsync(st->root, nullptr);
  cudaDeviceSynchronize();
  for (auto& w : st->wcache) cudaFreeAsync(w.W, nullptr);
  st->wcache.clear();
  cudaDeviceSynchronize();
  if (st->d_status) cudaFree(st->d_status);
  if (st->pinned) cudaFreeHost(st->pinned);
  delete st;
  return BHT_OK;
}

}  // extern "C"

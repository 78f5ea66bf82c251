"""Python binding of libbht (batch hierarchical Tucker on GB300).

Argument marshalling only: every step of BHT-l2r, HT-RISE and the
reconstruction runs inside libbht.so (include/bht.h). The binding turns
tensors into pointers, sizes and a stream handle, calls the C entry point of
the same name and raises on a non-zero status. There is no CPU fallback: if
the shared library is missing, importing this package raises.

Batches may be torch tensors (CUDA or CPU) or numpy arrays, float32 or
float64, C-contiguous, item-major [N, n_1, ..., n_d].
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbht.so")

BHT_OK = 0
BHT_F32, BHT_F64 = 0, 1
BHT_PREC_FP64, BHT_PREC_MIXED = 0, 1
STATUS_NAMES = {0: "BHT_OK", 1: "BHT_EINVAL", 2: "BHT_ENOMEM", 3: "BHT_ECAPACITY", 4: "BHT_ECUDA",
                5: "BHT_ENUMERIC", 6: "BHT_ETIMEOUT", 7: "BHT_EUNSUPPORTED"}
(BHT_EINVAL, BHT_ENOMEM, BHT_ECAPACITY, BHT_ECUDA, BHT_ENUMERIC, BHT_ETIMEOUT, BHT_EUNSUPPORTED) = range(1, 8)


class BHTError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("budget", ctypes.c_int32), ("predictor", ctypes.c_void_p),
                ("node_features", ctypes.c_void_p), ("node_labels", ctypes.c_void_p)]


class _Info(ctypes.Structure):
    _fields_ = [("skipped", ctypes.c_int32), ("batch_reads", ctypes.c_int32), ("eps_proj", ctypes.c_double),
                ("eps_des", ctypes.c_double), ("norm_y", ctypes.c_double), ("n_items_total", ctypes.c_int64),
                ("pred_nodes", ctypes.c_int32), ("pred_skipped", ctypes.c_int32), ("pred_fallback", ctypes.c_int32),
                ("pred_missed", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2412_16544_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "bht_tree_create_balanced": [i32, P(i64), P(vp)],
        "bht_tree_destroy": [vp],
        "bht_tree_info": [vp, P(i32), P(i32)],
        "bht_l2r": [vp, vp, i32, i64, dbl, P(_Opts), vp, P(vp)],
        "htrise_update": [vp, vp, i32, i64, dbl, P(_Opts), vp, P(_Info)],
        "htrise_update_stream": [vp, vp, i32, i64, i64, dbl, P(_Opts), vp, P(_Info), P(i64)],
        "ht_reconstruct": [vp, i64, i64, vp, i32, vp],
        "ht_encode": [vp, vp, i32, i64, vp, vp],
        "bht_get_ranks": [vp, P(i64), i64],
        "bht_get_dims": [vp, P(i32), P(i64), i64],
        "bht_get_core": [vp, i32, vp, i64, P(i64)],
        "bht_get_root": [vp, i64, i64, vp, i64],
        "bht_num_elements": [vp, P(i64)],
        "bht_state_destroy": [vp],
        "bht_launch_count": [P(i64), i32],
        "bht_batch_reads": [P(i64), i32],
        "bht_debug_withhold_barrier": [i32, i32],
        "bht_profile_enable": [ctypes.c_uint32],
        "bht_mode_product": [vp, i64, i64, vp, i64, i32, vp, i64, vp, vp],
        "bht_sym_eig": [vp, i64, vp, vp, i64, vp],
        "bht_mode_product_noalloc": [vp, i64, i64, vp, i64, vp, i64, vp, vp],
        "bht_profile_read": [P(dbl), P(i64), P(dbl), P(dbl), i32, i32],
        "ht_decode": [vp, vp, i64, vp, i32, vp],
        "ht_l2r": [i32, P(i64), vp, i32, i64, dbl, P(_Opts), vp, P(vp)],
        "ht_relative_test_error": [vp, vp, i32, i64, P(dbl), P(dbl), vp],
        "bht_normalize": [vp, i32, i64, i64, i32, vp, vp],
        "bht_denormalize": [vp, i32, i64, i64, vp, vp],
        "bht_permute_items": [vp, i32, i64, i32, P(i64), P(ctypes.c_int32), vp, vp],
        "bht_mlp_create": [i32, i32, vp, P(vp)],
        "bht_mlp_destroy": [vp],
        "bht_mlp_num_params": [vp, P(i64)],
        "bht_mlp_get_params": [vp, vp, i64, vp],
        "bht_mlp_forward": [vp, vp, i64, vp, vp],
        "bht_mlp_loss_grad": [vp, vp, vp, i64, P(dbl), vp],
        "bht_mlp_adam_step": [vp, dbl, vp],
        "bht_sketch_features": [vp, i64, dbl, dbl, ctypes.c_uint64, vp, vp],
        "bht_synth_chebyshev": [vp, i64, i32, i32, i32, i32, dbl, ctypes.c_uint64, i64, vp, vp],
        "bht_probe_fma_rate": [i32, P(dbl), vp],
        "bht_pair_gram": [vp, i64, i64, i64, i64, vp, vp, i32, vp],
        "bht_pair_project": [vp, i64, i64, i64, i64, vp, i64, vp, i64, vp, vp, vp],
        "bht_eig_min_above": [vp, i64, ctypes.c_double, ctypes.POINTER(i32), vp],
        "bht_sym_eig_small": [vp, i64, vp, vp, vp],
        "bht_tri_project": [vp, i64, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bht_last_error.restype = ctypes.c_char_p
    lib.bht_last_error.argtypes = []
    lib.bht_version.restype = ctypes.c_char_p
    lib.bht_version.argtypes = []
    lib.bht_kernel_class_name.restype = ctypes.c_char_p
    lib.bht_kernel_class_name.argtypes = [i32]
    return lib


_lib = _load()
EXPORTED = ["bht_tree_create_balanced", "bht_tree_destroy", "bht_tree_info", "bht_l2r", "htrise_update",
            "htrise_update_stream",
            "ht_reconstruct", "ht_encode", "bht_get_ranks", "bht_get_dims", "bht_get_core", "bht_get_root",
            "bht_num_elements", "bht_state_destroy", "bht_launch_count", "bht_last_error", "bht_version",
            "bht_profile_enable", "bht_profile_read", "bht_kernel_class_name", "bht_mode_product", "bht_sym_eig", "bht_sym_eig_small", "bht_eig_min_above",
            "bht_mode_product_noalloc",
            "bht_mlp_create", "bht_mlp_destroy", "bht_mlp_num_params", "bht_mlp_get_params", "bht_mlp_forward",
            "bht_mlp_loss_grad", "bht_mlp_adam_step", "bht_sketch_features", "ht_decode", "ht_l2r",
            "ht_relative_test_error", "bht_normalize", "bht_denormalize", "bht_permute_items",
            "bht_synth_chebyshev", "bht_probe_fma_rate", "bht_pair_gram", "bht_pair_project", "bht_tri_project",
            "bht_batch_reads",
            "bht_debug_withhold_barrier"]
KERNEL_CLASSES = 21


def _check(status: int, where: str):
    if status != BHT_OK:
        raise BHTError(status, where, _lib.bht_last_error().decode(errors="replace"))


def lib():
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _buffer(x):
    """(pointer, dtype code, shape, keepalive) of a torch tensor or numpy array."""
    torch = _torch()
    if torch is not None and isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("batch must be C-contiguous")
        if x.dtype == torch.float32:
            code = BHT_F32
        elif x.dtype == torch.float64:
            code = BHT_F64
        else:
            raise TypeError("batch must be float32 or float64")
        return ctypes.c_void_p(x.data_ptr()), code, tuple(x.shape), x
    a = np.asarray(x)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("batch must be C-contiguous")
    if a.dtype == np.float32:
        code = BHT_F32
    elif a.dtype == np.float64:
        code = BHT_F64
    else:
        raise TypeError("batch must be float32 or float64")
    return ctypes.c_void_p(a.ctypes.data), code, a.shape, a


def _stream(stream):
    if stream is None:
        torch = _torch()
        if torch is not None and torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _opts(precision, predictor=None, node_features=None, node_labels=None, budget=None):
    if precision is None and predictor is None and node_features is None and node_labels is None and budget is None:
        return None
    code = {"fp64": BHT_PREC_FP64, "mixed": BHT_PREC_MIXED, None: BHT_PREC_FP64}.get(precision, precision)
    bcode = {"uniform": 0, "adaptive": 1, None: -1}.get(budget, budget)  # -1: the state's own
    o = _Opts(int(code), int(bcode), predictor.value if predictor is not None else None,
              node_features.ctypes.data if node_features is not None else None,
              node_labels.ctypes.data if node_labels is not None else None)
    return ctypes.byref(o)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

@dataclass
class UpdateInfo:
    skipped: bool
    eps_proj: float
    eps_des: float
    norm_y: float
    n_items_total: int
    pred_nodes: int = 0
    pred_skipped: int = 0
    pred_fallback: int = 0
    pred_missed: int = 0
    batch_reads: int = 0


def bht_tree_create_balanced(dims) -> ctypes.c_void_p:
    arr = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    _check(_lib.bht_tree_create_balanced(len(dims), arr, ctypes.byref(h)), "bht_tree_create_balanced")
    return h


def bht_tree_destroy(tree) -> None:
    _check(_lib.bht_tree_destroy(tree), "bht_tree_destroy")


def bht_tree_info(tree):
    depth, nodes = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.bht_tree_info(tree, ctypes.byref(depth), ctypes.byref(nodes)), "bht_tree_info")
    return depth.value, nodes.value


def bht_l2r(tree, Y, eps_rel: float, precision=None, stream=None, budget=None) -> ctypes.c_void_p:
    """budget: "uniform" (default) or "adaptive" (App. C); also the default of later htrise_update calls."""
    ptr, code, shape, keep = _buffer(Y)
    h = ctypes.c_void_p()
    _check(_lib.bht_l2r(tree, ptr, code, int(shape[0]), float(eps_rel), _opts(precision, budget=budget),
                        _stream(stream), ctypes.byref(h)), "bht_l2r")
    del keep
    return h


def ht_l2r(Y, eps_rel: float, precision=None, stream=None) -> ctypes.c_void_p:
    """Plain HT baseline: the batch Y [N, n_1..n_d] as one tensor with the batch as the last leaf."""
    ptr, code, shape, keep = _buffer(Y)
    dims = (ctypes.c_int64 * (len(shape) - 1))(*shape[1:])
    h = ctypes.c_void_p()
    _check(_lib.ht_l2r(len(shape) - 1, dims, ptr, code, int(shape[0]), float(eps_rel), _opts(precision),
                       _stream(stream), ctypes.byref(h)), "ht_l2r")
    del keep
    return h


def htrise_update(state, Y, eps_rel: float, precision=None, stream=None, predictor=None, node_features=None,
                  node_labels=None, budget=None) -> UpdateInfo:
    """node_features (float32 [nodes][66]) and node_labels (int64 [nodes][2]): host numpy arrays the call
    fills for the nodes whose residual it forms (the predictor's training pairs)."""
    ptr, code, shape, keep = _buffer(Y)
    info = _Info()
    for a, dt in ((node_features, np.float32), (node_labels, np.int64)):
        if a is not None and (a.dtype != dt or not a.flags.c_contiguous):
            raise ValueError("node_features must be float32 and node_labels int64, C-contiguous")
    _check(_lib.htrise_update(state, ptr, code, int(shape[0]), float(eps_rel),
                              _opts(precision, predictor, node_features, node_labels, budget), _stream(stream),
                              ctypes.byref(info)), "htrise_update")
    del keep
    return UpdateInfo(bool(info.skipped), info.eps_proj, info.eps_des, info.norm_y, info.n_items_total,
                      info.pred_nodes, info.pred_skipped, info.pred_fallback, info.pred_missed, info.batch_reads)


def htrise_update_stream(state, Y, eps_rel: float, precision=None, stream=None, budget=None):
    """HT-RISE over the batches Y[0], Y[1], ... ([count][N][n_1]..[n_d], device or host, host ideally
    pinned) in one call, the next batch's projection overlapping the current batch's skip test.
    Returns the list of UpdateInfo, one per batch."""
    ptr, code, shape, keep = _buffer(Y)
    if len(shape) < 3:
        raise ValueError("Y must be [count][N][n_1]..[n_d]")
    count, n = int(shape[0]), int(shape[1])
    infos = (_Info * max(count, 1))()
    done = ctypes.c_int64()
    _check(_lib.htrise_update_stream(state, ptr, code, n, count, float(eps_rel),
                                     _opts(precision, None, None, None, budget), _stream(stream), infos,
                                     ctypes.byref(done)), "htrise_update_stream")
    del keep
    return [UpdateInfo(bool(i.skipped), i.eps_proj, i.eps_des, i.norm_y, i.n_items_total, i.pred_nodes,
                       i.pred_skipped, i.pred_fallback, i.pred_missed, i.batch_reads) for i in infos[:count]]


def bht_get_dims(state):
    d = ctypes.c_int32()
    dims = (ctypes.c_int64 * 16)()
    _check(_lib.bht_get_dims(state, ctypes.byref(d), dims, 16), "bht_get_dims")
    return [dims[i] for i in range(d.value)]


def bht_get_ranks(state):
    dims = bht_get_dims(state)
    n = 2 * len(dims) - 1
    out = (ctypes.c_int64 * n)()
    _check(_lib.bht_get_ranks(state, out, n), "bht_get_ranks")
    return [out[i] for i in range(n)]


def ht_reconstruct(state, first: int, count: int, out=None, dtype="float32", stream=None):
    """Decode items first..first+count-1 into `out` (allocated on the current CUDA device when None)."""
    dims = bht_get_dims(state)
    if out is None:
        torch = _torch()
        tdt = torch.float32 if dtype in ("float32", BHT_F32) else torch.float64
        out = torch.empty((count, *dims), dtype=tdt, device="cuda")
    ptr, code, _, keep = _buffer(out)
    _check(_lib.ht_reconstruct(state, int(first), int(count), ptr, code, _stream(stream)), "ht_reconstruct")
    return out


def ht_encode(state, Y, out=None, stream=None):
    ranks = bht_get_ranks(state)
    ptr, code, shape, keep = _buffer(Y)
    dims = bht_get_dims(state)
    if tuple(shape[1:]) != tuple(dims):
        raise ValueError(f"items must be [N, {', '.join(map(str, dims))}], got {tuple(shape)}")
    if out is None:
        out = np.empty((shape[0], ranks[1], ranks[2]), dtype=np.float64)
    optr, ocode, _, okeep = _buffer(out)
    if ocode != BHT_F64:
        raise TypeError("ht_encode writes float64")
    _check(_lib.ht_encode(state, ptr, code, int(shape[0]), optr, _stream(stream)), "ht_encode")
    return out


def ht_decode(state, Z, out=None, dtype="float32", stream=None):
    """Decode latent items Z ([N][r11][r12] float64, host or device) into `out` (device when None)."""
    ptr, code, shape, keep = _buffer(Z)
    if code != BHT_F64:
        raise TypeError("latent items are float64")
    ranks = bht_get_ranks(state)
    if len(shape) != 3 or tuple(shape[1:]) != (ranks[1], ranks[2]):
        raise ValueError(f"latent items must be [N, {ranks[1]}, {ranks[2]}], got {tuple(shape)}")
    dims = bht_get_dims(state)
    if out is None:
        torch = _torch()
        tdt = torch.float32 if dtype in ("float32", BHT_F32) else torch.float64
        out = torch.empty((shape[0], *dims), dtype=tdt, device="cuda")
    optr, ocode, oshape, okeep = _buffer(out)
    if tuple(oshape) != (shape[0], *dims):
        raise ValueError(f"out must be [{shape[0]}, {', '.join(map(str, dims))}], got {tuple(oshape)}")
    _check(_lib.ht_decode(state, ptr, int(shape[0]), optr, ocode, _stream(stream)), "ht_decode")
    del keep, okeep
    return out


def relative_test_error(state, X, per_item: bool = False, stream=None):
    """Mean over the items of X of ||X_i - decode(encode(X_i))|| / ||X_i|| (eq. generalization_performance);
    with per_item=True also the per-item errors."""
    ptr, code, shape, keep = _buffer(X)
    dims = bht_get_dims(state)
    if tuple(shape[1:]) != tuple(dims):
        raise ValueError(f"items must be [N, {', '.join(map(str, dims))}], got {tuple(shape)}")
    rte = ctypes.c_double()
    errs = np.zeros(shape[0], dtype=np.float64)
    _check(_lib.ht_relative_test_error(state, ptr, code, int(shape[0]), ctypes.byref(rte),
                                       errs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)),
           "ht_relative_test_error")
    del keep
    return (rte.value, errs) if per_item else rte.value


NORMALIZATIONS = {"none": 0, "maxabs": 1, "unitvec": 2, "zscore": 3}


def bht_normalize(Y, kind: str, groups: int = None, stream=None) -> np.ndarray:
    """Normalise the device tensor Y in place, group by group (default: one group per item); returns the
    (shift, scale) parameters [groups, 2]."""
    ptr, code, shape, keep = _buffer(Y)
    total = int(np.prod(shape)) if len(shape) else 0
    groups = int(shape[0]) if groups is None else int(groups)
    if groups <= 0 or total % groups:
        raise ValueError("groups must divide the element count")
    params = np.zeros((groups, 2), dtype=np.float64)
    _check(_lib.bht_normalize(ptr, code, groups, total // groups, NORMALIZATIONS[kind],
                              ctypes.c_void_p(params.ctypes.data), _stream(stream)), "bht_normalize")
    del keep
    return params


def bht_denormalize(Y, params, stream=None) -> None:
    ptr, code, shape, keep = _buffer(Y)
    params = np.ascontiguousarray(params, dtype=np.float64)
    groups = params.shape[0]
    total = int(np.prod(shape))
    if groups <= 0 or total % groups:
        raise ValueError("params rows must divide the element count")
    _check(_lib.bht_denormalize(ptr, code, groups, total // groups, ctypes.c_void_p(params.ctypes.data),
                                _stream(stream)), "bht_denormalize")
    del keep


def bht_permute_items(Y, perm, stream=None):
    """Items of the device tensor Y [N, n_1..n_d] with their axes reordered: out axis k = item axis perm[k]."""
    torch = _torch()
    ptr, code, shape, keep = _buffer(Y)
    d = len(shape) - 1
    perm = [int(p) for p in perm]
    if len(perm) != d:
        raise ValueError("perm needs one entry per item axis")
    out = torch.empty((shape[0], *[shape[1 + p] for p in perm]), dtype=Y.dtype, device=Y.device)
    optr, _, _, okeep = _buffer(out)
    dims = (ctypes.c_int64 * d)(*shape[1:])
    pm = (ctypes.c_int32 * d)(*perm)
    _check(_lib.bht_permute_items(ptr, code, int(shape[0]), d, dims, pm, optr, _stream(stream)), "bht_permute_items")
    del keep, okeep
    return out


def bht_get_core(state, node: int) -> np.ndarray:
    n = ctypes.c_int64()
    _check(_lib.bht_get_core(state, int(node), None, 0, ctypes.byref(n)), "bht_get_core")
    buf = np.empty(n.value, dtype=np.float64)
    _check(_lib.bht_get_core(state, int(node), ctypes.c_void_p(buf.ctypes.data), n.value, ctypes.byref(n)),
           "bht_get_core")
    return buf


def bht_get_root(state, first: int, count: int, out=None):
    """Root slices [count, r11, r12] as float64 in host memory: a new numpy array, or `out` (a numpy array
    or a CPU torch tensor, e.g. pinned, of that shape)."""
    ranks = bht_get_ranks(state)
    if out is None:
        out = np.empty((count, ranks[1], ranks[2]), dtype=np.float64)
    ptr, code, shape, keep = _buffer(out)
    if code != BHT_F64 or tuple(shape) != (count, ranks[1], ranks[2]):
        raise ValueError(f"out must be float64 [{count}, {ranks[1]}, {ranks[2]}]")
    _check(_lib.bht_get_root(state, int(first), int(count), ptr, int(np.prod(shape))), "bht_get_root")
    del keep
    return out


def bht_num_elements(state) -> int:
    n = ctypes.c_int64()
    _check(_lib.bht_num_elements(state, ctypes.byref(n)), "bht_num_elements")
    return n.value


def bht_state_destroy(state) -> None:
    _check(_lib.bht_state_destroy(state), "bht_state_destroy")


def bht_launch_count(reset: bool = False) -> int:
    n = ctypes.c_int64()
    _check(_lib.bht_launch_count(ctypes.byref(n), 1 if reset else 0), "bht_launch_count")
    return n.value


def bht_batch_reads(reset: bool = False) -> int:
    """Kernels of this thread's compression calls that read a whole input batch, since the last reset."""
    n = ctypes.c_int64()
    _check(_lib.bht_batch_reads(ctypes.byref(n), 1 if reset else 0), "bht_batch_reads")
    return n.value


def bht_debug_withhold_barrier(launches: int, wait_ms: int = 20) -> None:
    """Arm the timeout-path test: the next `launches` multi-CTA tridiagonalisations withhold one grid-barrier
    arrival and give up their waits after wait_ms (the call then fails with BHT_ETIMEOUT)."""
    _check(_lib.bht_debug_withhold_barrier(int(launches), int(wait_ms)), "bht_debug_withhold_barrier")


def bht_mode_product(X, U, S: int, precision="mixed", R2: int = 1, out=None, norms=None, stream=None):
    """out[(o S + s) R2 + i] = sum_k X[o R2 + i, k] U[k, s] on device tensors (X fp32 [rows, K], U fp64 [K, S])."""
    torch = _torch()
    rows, K = X.shape
    if out is None:
        out = torch.empty(rows * S, dtype=torch.float32, device=X.device)
    code = {"fp64": BHT_PREC_FP64, "mixed": BHT_PREC_MIXED}.get(precision, precision)
    nptr = ctypes.c_void_p(norms.data_ptr()) if norms is not None else None
    _check(_lib.bht_mode_product(ctypes.c_void_p(X.data_ptr()), rows, K, ctypes.c_void_p(U.data_ptr()), int(S),
                                 int(code), ctypes.c_void_p(out.data_ptr()), int(R2), nptr, _stream(stream)),
           "bht_mode_product")
    return out


def bht_mode_product_noalloc(X, U, S: int, R2: int = 1, out=None, norms=None, stream=None):
    """bht_mode_product (tensor cores) with the library allocating nothing: out must be given by the caller."""
    torch = _torch()
    if out is None:
        raise ValueError("bht_mode_product_noalloc writes into a caller-owned output")
    if X.dim() != 2:
        raise ValueError("X must be [rows, K]")
    rows, K = X.shape
    for name, t, dt in (("X", X, torch.float32), ("U", U, torch.float64), ("out", out, torch.float32)):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor")
    if U.dim() != 2 or U.shape[0] != K or U.shape[1] != S:
        raise ValueError(f"U must be [{K}, {S}]")
    if out.numel() < rows * S:
        raise ValueError(f"out holds {out.numel()} elements, the product needs {rows * S}")
    if norms is not None and not (norms.is_cuda and norms.dtype == torch.float64 and norms.is_contiguous()
                                  and norms.numel() >= 2):
        raise ValueError("norms must be a contiguous float64 CUDA tensor of at least 2 elements")
    nptr = ctypes.c_void_p(norms.data_ptr()) if norms is not None else None
    _check(_lib.bht_mode_product_noalloc(ctypes.c_void_p(X.data_ptr()), rows, K, ctypes.c_void_p(U.data_ptr()),
                                         int(S), ctypes.c_void_p(out.data_ptr()), int(R2), nptr, _stream(stream)),
           "bht_mode_product_noalloc")
    return out


def bht_pair_gram(X, tensor_cores=False, stream=None):
    """Gram matrices of modes 1 and 2 of a contiguous fp32 CUDA tensor X [A, na, nb, B] (one read of X);
    tensor_cores: the split-TF32 tensor-core pass where the shape has one (24 x 24), else FP32 SIMT."""
    torch = _torch()
    A, na, nb, B = X.shape
    Ga = torch.empty((na, na), dtype=torch.float64, device=X.device)
    Gb = torch.empty((nb, nb), dtype=torch.float64, device=X.device)
    _check(_lib.bht_pair_gram(ctypes.c_void_p(X.data_ptr()), A, na, nb, B, ctypes.c_void_p(Ga.data_ptr()),
                              ctypes.c_void_p(Gb.data_ptr()), 1 if tensor_cores else 0, _stream(stream)),
           "bht_pair_gram")
    return Ga, Gb


def bht_pair_project(X, Ua, Ub, norms=None, stream=None):
    """X [A, na, nb, B] x_1 Ua^T x_2 Ub^T -> [A, ra, rb, B] (fp32 CUDA X, FP64 CUDA bases)."""
    torch = _torch()
    A, na, nb, B = X.shape
    ra, rb = Ua.shape[1], Ub.shape[1]
    out = torch.empty((A, ra, rb, B), dtype=torch.float32, device=X.device)
    nptr = ctypes.c_void_p(norms.data_ptr()) if norms is not None else None
    _check(_lib.bht_pair_project(ctypes.c_void_p(X.data_ptr()), A, na, nb, B, ctypes.c_void_p(Ua.data_ptr()), ra,
                                 ctypes.c_void_p(Ub.data_ptr()), rb, ctypes.c_void_p(out.data_ptr()), nptr,
                                 _stream(stream)), "bht_pair_project")
    return out


def bht_tri_project(X, U1, U2, U3, norms=None, stream=None):
    """X [A, n1, n2, n3] x_1 U1^T x_2 U2^T x_3 U3^T -> [A, r1, r2, r3] (fp32 CUDA X, FP64 CUDA bases)."""
    torch = _torch()
    A, n1, n2, n3 = X.shape
    r1, r2, r3 = U1.shape[1], U2.shape[1], U3.shape[1]
    out = torch.empty((A, r1, r2, r3), dtype=torch.float32, device=X.device)
    nptr = ctypes.c_void_p(norms.data_ptr()) if norms is not None else None
    _check(_lib.bht_tri_project(ctypes.c_void_p(X.data_ptr()), A, n1, n2, n3, ctypes.c_void_p(U1.data_ptr()), r1,
                                ctypes.c_void_p(U2.data_ptr()), r2, ctypes.c_void_p(U3.data_ptr()), r3,
                                ctypes.c_void_p(out.data_ptr()), nptr, _stream(stream)), "bht_tri_project")
    return out


def bht_sym_eig(G, r: int, stream=None):
    """Eigenvalues (descending) and the r leading eigenvectors of a symmetric fp64 CUDA tensor G (overwritten)."""
    torch = _torch()
    n = G.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device=G.device)
    U = torch.empty((n, max(r, 1)), dtype=torch.float64, device=G.device)
    _check(_lib.bht_sym_eig(ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(lam.data_ptr()),
                            ctypes.c_void_p(U.data_ptr()), int(r), _stream(stream)), "bht_sym_eig")
    return lam, U[:, :r]


def bht_sym_eig_small(G, stream=None):
    """Ritz values (decreasing) and orthonormal vectors of a symmetric fp64 CUDA tensor G, n <= 32
    (FP32 Jacobi, FP64 Newton-Schulz and Ritz values; G is not written)."""
    torch = _torch()
    if G.dtype != torch.float64 or not G.is_cuda or G.dim() != 2 or G.shape[0] != G.shape[1]:
        raise ValueError("G must be a square float64 CUDA tensor")
    G = G.contiguous()
    n = G.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device=G.device)
    V = torch.empty((n, n), dtype=torch.float64, device=G.device)
    _check(_lib.bht_sym_eig_small(ctypes.c_void_p(G.data_ptr()), n, ctypes.c_void_p(lam.data_ptr()),
                                  ctypes.c_void_p(V.data_ptr()), _stream(stream)), "bht_sym_eig_small")
    return lam, V


def bht_eig_min_above(G, tau: float, stream=None) -> bool:
    """True when a Cholesky factorisation certifies that every eigenvalue of the symmetric fp64 CUDA
    tensor G exceeds tau (G is not written)."""
    torch = _torch()
    if G.dtype != torch.float64 or not G.is_cuda or G.dim() != 2 or G.shape[0] != G.shape[1]:
        raise ValueError("G must be a square float64 CUDA tensor")
    G = G.contiguous()
    v = ctypes.c_int32(0)
    _check(_lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), G.shape[0], float(tau), ctypes.byref(v),
                                  _stream(stream)), "bht_eig_min_above")
    return v.value == 1


def bht_probe_fma_rate(dtype: str = "float64", stream=None) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s for "float64" or "float32"."""
    v = ctypes.c_double()
    code = BHT_F64 if dtype in ("float64", BHT_F64) else BHT_F32
    _check(_lib.bht_probe_fma_rate(code, ctypes.byref(v), _stream(stream)), "bht_probe_fma_rate")
    return v.value


def bht_profile_enable(class_mask: int) -> None:
    _check(_lib.bht_profile_enable(int(class_mask)), "bht_profile_enable")


def bht_profile_read(reset: bool = False, work: bool = False) -> dict:
    """Per kernel class: (ms, launches) or, with work=True, (ms, launches, flops, bytes)."""
    ms = (ctypes.c_double * KERNEL_CLASSES)()
    n = (ctypes.c_int64 * KERNEL_CLASSES)()
    fl = (ctypes.c_double * KERNEL_CLASSES)()
    by = (ctypes.c_double * KERNEL_CLASSES)()
    _check(_lib.bht_profile_read(ms, n, fl, by, KERNEL_CLASSES, 1 if reset else 0), "bht_profile_read")
    names = [bht_kernel_class_name(i) for i in range(KERNEL_CLASSES)]
    if work:
        return {names[i]: (ms[i], n[i], fl[i], by[i]) for i in range(KERNEL_CLASSES) if names[i] != "?"}
    return {names[i]: (ms[i], n[i]) for i in range(KERNEL_CLASSES) if names[i] != "?"}


def bht_kernel_class_name(cls: int) -> str:
    return _lib.bht_kernel_class_name(int(cls)).decode()


def bht_version() -> str:
    return _lib.bht_version().decode()


def bht_last_error() -> str:
    return _lib.bht_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# rank / expansion predictor
# ---------------------------------------------------------------------------

def bht_mlp_create(params, f_in: int = 66, hidden: int = 128) -> ctypes.c_void_p:
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(_lib.bht_mlp_create(int(f_in), int(hidden), ctypes.c_void_p(p.ctypes.data), ctypes.byref(h)),
           "bht_mlp_create")
    return h


def bht_mlp_destroy(net) -> None:
    _check(_lib.bht_mlp_destroy(net), "bht_mlp_destroy")


def bht_mlp_num_params(net) -> int:
    n = ctypes.c_int64()
    _check(_lib.bht_mlp_num_params(net, ctypes.byref(n)), "bht_mlp_num_params")
    return n.value


def bht_mlp_get_params(net, grad: bool = False):
    n = bht_mlp_num_params(net)
    p = np.empty(n, dtype=np.float32)
    g = np.empty(n, dtype=np.float32) if grad else None
    _check(_lib.bht_mlp_get_params(net, ctypes.c_void_p(p.ctypes.data), n,
                                   ctypes.c_void_p(g.ctypes.data) if grad else None), "bht_mlp_get_params")
    return (p, g) if grad else p


def bht_mlp_forward(net, X, stream=None) -> np.ndarray:
    ptr, code, shape, keep = _buffer(X)
    if code != BHT_F32:
        raise ValueError("predictor inputs are float32")
    out = np.empty((shape[0], 2), dtype=np.float32)
    _check(_lib.bht_mlp_forward(net, ptr, int(shape[0]), ctypes.c_void_p(out.ctypes.data), _stream(stream)),
           "bht_mlp_forward")
    del keep
    return out


def bht_mlp_loss_grad(net, X, T, stream=None) -> float:
    px, cx, sx, kx = _buffer(X)
    pt, ct, st_, kt = _buffer(T)
    if cx != BHT_F32 or ct != BHT_F32:
        raise ValueError("predictor inputs and targets are float32")
    loss = ctypes.c_double()
    _check(_lib.bht_mlp_loss_grad(net, px, pt, int(sx[0]), ctypes.byref(loss), _stream(stream)), "bht_mlp_loss_grad")
    del kx, kt
    return loss.value


def bht_mlp_adam_step(net, lr: float, stream=None) -> None:
    _check(_lib.bht_mlp_adam_step(net, float(lr), _stream(stream)), "bht_mlp_adam_step")


def bht_sketch_features(G, tol: float, norm: float, seed: int = 0, stream=None) -> np.ndarray:
    ptr, code, shape, keep = _buffer(G)
    if code != BHT_F64:
        raise ValueError("G is float64")
    f = np.empty(66, dtype=np.float32)
    _check(_lib.bht_sketch_features(ptr, int(shape[0]), float(tol), float(norm), int(seed),
                                    ctypes.c_void_p(f.ctypes.data), _stream(stream)), "bht_sketch_features")
    del keep
    return f


def bht_synth_chebyshev(coeffs, n: int, seed: int, first_item: int, noise_std: float = 0.01, out=None,
                        stream=None):
    """Items of the Chebyshev sensor stream drawn on the device from coefficients [count, terms, d, degree + 1]
    (float64, host or device); returns (or fills) a float32 CUDA tensor [count] + [n] * d."""
    torch = _torch()
    ptr, code, shape, keep = _buffer(coeffs)
    if code != BHT_F64 or len(shape) != 4:
        raise ValueError("coefficients are float64 [count, terms, d, degree + 1]")
    count, terms, d, deg1 = (int(x) for x in shape)
    if out is None:
        out = torch.empty((count,) + (n,) * d, dtype=torch.float32, device="cuda")
    if not (out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == count * n ** d):
        raise ValueError(f"out must be a contiguous float32 CUDA tensor of {count * n ** d} elements")
    _check(_lib.bht_synth_chebyshev(ptr, count, int(n), d, terms, deg1 - 1, float(noise_std), int(seed),
                                    int(first_item), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "bht_synth_chebyshev")
    del keep
    return out

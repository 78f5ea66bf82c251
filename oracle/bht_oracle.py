"""FP64 CPU oracle of the batch hierarchical Tucker method (BHT-l2r and HT-RISE).

Test infrastructure only: ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it. The GPU library neither imports nor
links it; the two share no code.

Notation follows the paper: a batch of ``N`` items with ``d`` non-batch modes
``n_1..n_d``; a dimension tree ``T`` over modes 1..d only (the batch is carried
by the root, Section 3.1); layers ``l = 0`` (root) .. ``p``; HT ranks
``r_{l,i}``; relative tolerance ``eps_rel``.

Layout: internally the oracle follows the paper and keeps the batch LAST
(``[n_1, ..., n_d, N]``, Section 3.1). The public functions take and return
item-major arrays ``[N, n_1, ..., n_d]`` and transpose at the boundary; the
footnote to Section 3.1 states the batch position does not matter.

Every SVD is ``numpy.linalg.svd`` of an explicit unfolding, in float64.

Readings of the paper where it is silent, garbled or self-inconsistent
(each applied below where it matters):

R1  Truncation rule (eq. ht_leaf_svd, eq. svd_on_residual): keep the smallest
    r with sum_{i>r} sigma_i^2 <= eps_nw^2. BHT-l2r nodes keep r >= 1; the
    residual truncation of HT-RISE may keep r_R = 0.
R2  Node-wise tolerance eps_nw = eps_abs / sqrt(2d-2) (Algorithm 1, Algorithm 2,
    Corollary bht_leaves_to_root), d = number of non-batch modes.
R3  Dimension tree: balanced binary over modes 1..d, the first child of a node
    with m modes takes ceil(m/2) of them (Fig. 2 left: {1,2,3},{4,5}).
R4  Reshape merge order (eq. ht_index_set_construction): C-order, the merged
    index of a transfer node is i_left * r_right + i_right; a transfer core is
    reshape(U, [r_left, r_right, r]) in the same order (eq. ht_tucker_core_reshape).
R5  HT-RISE eps_des = eps_rel * ||Y^k|| of the new batch (Algorithm 2).
R6  Algorithm 2 unfolds "mode l" at layer l: read as the mode of node j.
R7  eq. compute_residual builds U^{k-1} of a transfer node from the already
    zero-padded core, reshaped to [alpha, r^{k-1}] with alpha = product of the
    children's current ranks.
R8  The root is zero-padded in modes 1 and 2 before the new batch is appended
    (eq. incremental_zero_padding1 applied with l = 1; Theorem hit_past_stream).
R9  The new directions U_R are orthogonal to U^{k-1} "by definition"
    (eq. concatenating_orthonormal_vectors); the oracle still applies two
    Gram-Schmidt passes and a QR to U_R, a no-op in exact arithmetic.
R10 Leaves on a layer l < p are truncated and contracted at their own layer,
    from the partially projected intermediate of that layer (Algorithm 1).
R11 Reconstruction (eq. htucker_reconstruction) contracts the root with the two
    distinct layer-1 cores G_{1,1}, G_{1,2} (the printed G_{1,1}, G_{1,1} is a typo).
R12 In the skip test of Algorithm 2, ||Y||^2 - ||C||^2 is clamped at 0 before
    the square root.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# Dimension tree (Section 2.3, Fig. 2; reading R3)
# ---------------------------------------------------------------------------

class Node:
    """One node of the dimension tree: N_{l,i} = (successors, parent) of Section 2.3."""

    def __init__(self, nid: int, layer: int, modes: tuple, parent):
        self.id = nid            # breadth-first position, root = 0
        self.layer = layer
        self.modes = modes       # 0-based modes covered by the node
        self.parent = parent     # node id, None for the root
        self.children: list = []  # successor ids, ordered by position in their layer
        self.slot = None         # 0 / 1: which successor of the parent (t - 1 in padWithZeros)

    @property
    def is_leaf(self) -> bool:
        return not self.children

    @property
    def mode(self) -> int:
        assert self.is_leaf
        return self.modes[0]


class Tree:
    """Balanced binary dimension tree over modes 0..d-1 (batch excluded)."""

    def __init__(self, dims):
        dims = tuple(int(x) for x in dims)
        if len(dims) < 2:
            raise ValueError("the batch hierarchical Tucker format needs d >= 2 modes")
        self.dims = dims
        self.d = len(dims)
        self.nodes: list = []
        self.layers: list = []
        root = Node(0, 0, tuple(range(self.d)), None)
        self.nodes.append(root)
        frontier = [root]
        while frontier:
            self.layers.append([nd.id for nd in frontier])
            nxt = []
            for nd in frontier:
                m = len(nd.modes)
                if m == 1:
                    continue
                h = (m + 1) // 2  # first child takes ceil(m/2) modes
                for slot, modes in enumerate((nd.modes[:h], nd.modes[h:])):
                    ch = Node(len(self.nodes), nd.layer + 1, modes, nd.id)
                    ch.slot = slot
                    self.nodes.append(ch)
                    nd.children.append(ch.id)
                    nxt.append(ch)
            frontier = nxt
        self.p = len(self.layers) - 1
        self.leaf_of_mode = {nd.mode: nd.id for nd in self.nodes if nd.is_leaf}

    def layer_nodes(self, layer: int):
        return [self.nodes[i] for i in self.layers[layer]]

    def non_root(self):
        return self.nodes[1:]


def dimension_tree(dims) -> Tree:
    return Tree(dims)


# ---------------------------------------------------------------------------
# Elementary tensor operations (Section 2.1)
# ---------------------------------------------------------------------------

def unfold(C: np.ndarray, axis: int) -> np.ndarray:
    """Mode-`axis` matricization: that axis becomes the rows (Section 2.1)."""
    return np.moveaxis(C, axis, 0).reshape(C.shape[axis], -1)


def mode_product_t(C: np.ndarray, axis: int, U: np.ndarray) -> np.ndarray:
    """C x_axis U^T: contract axis `axis` (size n) with U (n x r); the axis keeps its place."""
    out = np.tensordot(C, U, axes=([axis], [0]))  # new axis (r) last
    return np.moveaxis(out, -1, axis)


def truncation_rank(s2: np.ndarray, eps_nw2: float, rmin: int) -> int:
    """Smallest r >= rmin with sum_{i >= r} s2[i] <= eps_nw2 (reading R1); s2 descending."""
    s2 = np.asarray(s2, dtype=np.float64)
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])  # tail[r] = sum_{i>=r} s2[i]
    r = int(np.nonzero(tail <= eps_nw2)[0][0])
    return min(max(r, rmin), len(s2)) if len(s2) else 0


def truncated_left_svd(M: np.ndarray, eps_nw: float, rmin: int = 1):
    """Error-truncated SVD keeping the left singular vectors (eq. ht_leaf_svd).

    Returns (U, s2): U with r orthonormal columns, s2 all squared singular values.
    """
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    s2 = s * s
    r = truncation_rank(s2, eps_nw * eps_nw, rmin)
    return U[:, :r].copy(), s2


def _orthogonalize_against(U_R: np.ndarray, U_old: np.ndarray) -> np.ndarray:
    """Reading R9: two classical Gram-Schmidt passes against U_old, then a QR with positive diagonal."""
    if U_R.shape[1] == 0:
        return U_R
    for _ in range(2):
        U_R = U_R - U_old @ (U_old.T @ U_R)
    Q, Rf = np.linalg.qr(U_R)
    sgn = np.sign(np.diag(Rf))
    sgn[sgn == 0] = 1.0
    return Q * sgn


# ---------------------------------------------------------------------------
# State of the batch-HT representation (Section 3.1, Fig. htucker_batch_new)
# ---------------------------------------------------------------------------

@dataclass
class BHTState:
    tree: Tree
    eps_rel: float
    cores: dict = field(default_factory=dict)   # leaf id -> U [n, r]; transfer id -> G [r_l, r_r, r]
    root: np.ndarray = None                     # G_0 [r_11, r_12, N_total] (batch last)
    n_items: int = 0
    budget: str = "uniform"                     # "uniform" (Algorithms 1, 2) or "adaptive" (App. C)

    def rank(self, nid: int) -> int:
        return self.cores[nid].shape[-1]

    def ranks(self) -> list:
        """[N_total] + [r of every non-root node, breadth-first order]."""
        return [self.n_items] + [self.rank(nd.id) for nd in self.tree.non_root()]

    def basis(self, nid: int) -> np.ndarray:
        """Orthonormal matrix form of a core: leaf U, or transfer G reshaped [alpha, r] (R4, R7)."""
        G = self.cores[nid]
        return G if G.ndim == 2 else G.reshape(-1, G.shape[-1])

    def root_items(self) -> np.ndarray:
        """The root core item-major, [N_total, r_11, r_12]."""
        return np.moveaxis(self.root, -1, 0)

    def num_elements(self) -> int:
        return int(sum(c.size for c in self.cores.values()) + self.root.size)


@dataclass
class UpdateInfo:
    skipped: bool
    eps_proj: float
    eps_des: float
    ranks_before: list
    ranks_after: list


def layer_shape(state: BHTState, layer: int) -> list:
    """Index set of a layer without the batch (eq. ht_index_set_construction, updateIndexSet)."""
    tree = state.tree
    out = []
    for nd in tree.layer_nodes(layer):
        if nd.is_leaf:
            out.append(tree.dims[nd.mode])
        else:
            a, b = nd.children
            out.append(state.rank(a) * state.rank(b))
    return out


def _reshape_to_layer(tree: Tree, C: np.ndarray, axes: list, layer: int):
    """Merge the projected axes of layer+1 into the index set of `layer` (eq. ht_index_set_construction).

    `axes` lists, for each non-batch axis of C, the node whose index it carries.
    A transfer node of `layer` merges its two children's adjacent axes in C-order (R4);
    a leaf of `layer` keeps its own axis.
    """
    shape, new_axes, pos = [], [], 0
    for nd in tree.layer_nodes(layer):
        if nd.is_leaf:
            assert axes[pos] == nd.id
            shape.append(C.shape[pos])
            pos += 1
        else:
            a, b = nd.children
            assert axes[pos] == a and axes[pos + 1] == b
            shape.append(C.shape[pos] * C.shape[pos + 1])
            pos += 2
        new_axes.append(nd.id)
    assert pos == len(axes)
    return C.reshape(shape + [C.shape[-1]]), new_axes


def _initial_axes(tree: Tree) -> list:
    return [tree.leaf_of_mode[m] for m in range(tree.d)]


def _to_paper_layout(Y: np.ndarray, tree: Tree) -> np.ndarray:
    Y = np.asarray(Y, dtype=np.float64)
    if Y.shape[1:] != tree.dims:
        raise ValueError(f"batch shape {Y.shape} does not match dims {tree.dims}")
    return np.moveaxis(Y, 0, -1)


# ---------------------------------------------------------------------------
# Algorithm 1: BHT-l2r
# ---------------------------------------------------------------------------

def _svds_above(tree: Tree, layer: int) -> int:
    """Number of truncations (non-root nodes) on the layers above `layer` (ell - 1 .. 1)."""
    return sum(len(tree.layers[l]) for l in range(1, layer))


def _adaptive_eps_nw(eps_abs2: float, norm2: float, C: np.ndarray, svd_rem: int) -> float:
    """App. C: the error spent so far eps_l^2 = ||Y||^2 - ||C_l||^2, the remaining budget
    eps_rem = sqrt(eps_abs^2 - eps_l^2), spread over the svd_rem truncations still to come."""
    eps_l2 = max(norm2 - float(np.sum(C * C)), 0.0)
    eps_rem2 = max(eps_abs2 - eps_l2, 0.0)
    return math.sqrt(eps_rem2 / svd_rem)


def bht_l2r(Y: np.ndarray, eps_rel: float, tree: Tree = None, budget: str = "uniform") -> BHTState:
    """Error-truncated leaves-to-root batch HT decomposition (Algorithm 1).

    Y: item-major batch [N, n_1, ..., n_d]. budget "uniform": eps_nw = eps_abs / sqrt(2d - 2) at every
    node (Algorithm 1); "adaptive": after each layer the error actually spent is measured and the
    remaining budget is spread over the remaining truncations (App. C).
    """
    if tree is None:
        tree = Tree(Y.shape[1:])
    C = _to_paper_layout(Y, tree)
    d, p = tree.d, tree.p
    state = BHTState(tree=tree, eps_rel=float(eps_rel), budget=budget)
    norm2 = float(np.sum(C * C))
    eps_nw = eps_rel * math.sqrt(norm2) / math.sqrt(2 * d - 2)   # node-wise tolerance (R2)
    axes = _initial_axes(tree)
    for layer in range(p, 0, -1):
        if layer < p:
            C, axes = _reshape_to_layer(tree, C, axes, layer)
            if budget == "adaptive":
                eps_nw = _adaptive_eps_nw(eps_rel * eps_rel * norm2, norm2, C, _svds_above(tree, layer + 1))
        # HOSVD of the layer: every node truncated from the same intermediate (R10)
        bases = {}
        for nd in tree.layer_nodes(layer):
            U, _ = truncated_left_svd(unfold(C, axes.index(nd.id)), eps_nw, rmin=1)
            bases[nd.id] = U
        for nd in tree.layer_nodes(layer):
            U = bases[nd.id]
            if nd.is_leaf:
                state.cores[nd.id] = U
            else:  # fold into a 3-way transfer core (eq. ht_tucker_core_reshape)
                a, b = nd.children
                state.cores[nd.id] = U.reshape(state.rank(a), state.rank(b), U.shape[1])
            C = mode_product_t(C, axes.index(nd.id), U)
    state.root = C.copy()        # G_0 = reshape(C, [r_11, r_12, N])
    state.n_items = C.shape[-1]
    return state


# ---------------------------------------------------------------------------
# Plain HT baseline: leaves-to-root HT (Sec. 2.3.1) with the batch as a leaf (Fig. htucker_as_node)
# ---------------------------------------------------------------------------

def ht_l2r(Y: np.ndarray, eps_rel: float) -> BHTState:
    """One-shot leaves-to-root HT decomposition of the N items as a single tensor (n_1, .., n_d, N): the
    batch is the last leaf of the balanced tree over d + 1 modes. Layers p .. 2 are truncated node by
    node from the same intermediate as in Algorithm 1; layer 1 is one error-truncated SVD of the matrix
    C_1 (eq. ht_last_svd) whose left and right singular vectors become the two layer-1 cores and whose
    singular values the root. Node-wise tolerance eps_rel ||Y|| / sqrt(2 (d + 1) - 3) (Theorem
    ht_nodewise_error). The state holds one item (root [r_11, r_12, 1], diagonal)."""
    T = np.moveaxis(np.asarray(Y, dtype=np.float64), 0, -1)
    tree = Tree(T.shape)
    C = T[..., None]             # a trailing axis of one item, so the layer helpers above apply
    state = BHTState(tree=tree, eps_rel=float(eps_rel))
    norm2 = float(np.sum(C * C))
    eps_nw = eps_rel * math.sqrt(norm2) / math.sqrt(2 * tree.d - 3)
    axes = _initial_axes(tree)

    def store(nd, U):
        if nd.is_leaf:
            state.cores[nd.id] = U
        else:
            a, b = nd.children
            state.cores[nd.id] = U.reshape(state.rank(a), state.rank(b), U.shape[1])

    for layer in range(tree.p, 1, -1):
        if layer < tree.p:
            C, axes = _reshape_to_layer(tree, C, axes, layer)
        bases = {nd.id: truncated_left_svd(unfold(C, axes.index(nd.id)), eps_nw, rmin=1)[0]
                 for nd in tree.layer_nodes(layer)}
        for nd in tree.layer_nodes(layer):
            store(nd, bases[nd.id])
            C = mode_product_t(C, axes.index(nd.id), bases[nd.id])
    C, axes = _reshape_to_layer(tree, C, axes, 1)
    U, s, Vt = np.linalg.svd(C[:, :, 0], full_matrices=False)
    r = truncation_rank(s * s, eps_nw * eps_nw, 1)
    left, right = tree.layer_nodes(1)
    store(left, U[:, :r].copy())
    store(right, Vt[:r].T.copy())
    state.root = np.diag(s[:r])[:, :, None]
    state.n_items = 1
    return state


def ht_items(state: BHTState) -> np.ndarray:
    """The tensor of a plain HT state back in item-major order [N, n_1, .., n_d]."""
    return np.moveaxis(reconstruct(state)[0], -1, 0)


# ---------------------------------------------------------------------------
# Step 1 of Algorithm 2: projection onto the existing cores
# ---------------------------------------------------------------------------

def _project_paper(state: BHTState, C: np.ndarray) -> np.ndarray:
    tree = state.tree
    axes = _initial_axes(tree)
    for layer in range(tree.p, 0, -1):
        if layer < tree.p:
            C, axes = _reshape_to_layer(tree, C, axes, layer)
        for nd in tree.layer_nodes(layer):
            C = mode_product_t(C, axes.index(nd.id), state.basis(nd.id))
    return C  # [r_11, r_12, N]


def project(state: BHTState, Y: np.ndarray) -> np.ndarray:
    """Latent representation of a batch on the current cores, item-major [N, r_11, r_12]."""
    return np.moveaxis(_project_paper(state, _to_paper_layout(Y, state.tree)), -1, 0)


# ---------------------------------------------------------------------------
# Algorithm 2: HT-RISE
# ---------------------------------------------------------------------------

def _pad_axis(A: np.ndarray, axis: int, extra: int) -> np.ndarray:
    """Concatenate `extra` zeros along `axis` (eq. concatenation with a zero tensor = padding)."""
    if extra == 0:
        return A
    shape = list(A.shape)
    shape[axis] = extra
    return np.concatenate([A, np.zeros(shape, dtype=A.dtype)], axis=axis)


def htrise_update(state: BHTState, Y: np.ndarray, eps_rel: float = None, budget: str = None) -> UpdateInfo:
    """Incremental update of the batch-HT state with a new batch (Algorithm 2). Mutates `state`.
    budget: as for bht_l2r (default: the state's)."""
    if eps_rel is None:
        eps_rel = state.eps_rel
    if budget is None:
        budget = state.budget
    tree = state.tree
    d, p = tree.d, tree.p
    Yp = _to_paper_layout(Y, tree)
    ranks_before = state.ranks()
    normY = np.linalg.norm(Yp)
    eps_des = eps_rel * normY                                   # R5
    Cbar = _project_paper(state, Yp)                            # Step 1
    eps_proj = math.sqrt(max(normY ** 2 - np.linalg.norm(Cbar) ** 2, 0.0))   # eq. relative_error_threshold, R12
    if eps_proj <= eps_des:
        # skip: every core but the root stays as it is
        state.root = np.concatenate([state.root, Cbar], axis=2)
        state.n_items += Cbar.shape[-1]
        return UpdateInfo(True, eps_proj, eps_des, ranks_before, state.ranks())

    eps_nw = eps_des / math.sqrt(2 * d - 2)
    C = Yp
    axes = _initial_axes(tree)
    root_pad = [0, 0]
    for layer in range(p, 0, -1):
        if layer < p:
            C, axes = _reshape_to_layer(tree, C, axes, layer)      # index set I^k of this layer
            if budget == "adaptive":
                eps_nw = _adaptive_eps_nw(eps_des * eps_des, normY ** 2, C, _svds_above(tree, layer + 1))
        # Steps 2-3 for every node of the layer, all from the same C
        new_bases = {}
        for nd in tree.layer_nodes(layer):
            M = unfold(C, axes.index(nd.id))
            U_old = state.basis(nd.id)                            # R7: padded core, reshaped
            R = M - U_old @ (U_old.T @ M)                         # eq. compute_residual
            U_R, _ = truncated_left_svd(R, eps_nw, rmin=0)        # eq. svd_on_residual
            U_R = U_R[:, :max(0, U_old.shape[0] - U_old.shape[1])]
            U_R = _orthogonalize_against(U_R, U_old)              # R9
            new_bases[nd.id] = (np.hstack([U_old, U_R]), U_R.shape[1])
        for nd in tree.layer_nodes(layer):
            U_new, r_R = new_bases[nd.id]
            # expandCore: append, then fold a transfer core back to 3-way
            if nd.is_leaf:
                state.cores[nd.id] = U_new
            else:
                a, b = nd.children
                state.cores[nd.id] = U_new.reshape(state.rank(a), state.rank(b), U_new.shape[1])
            # padWithZeros on the parent, in the mode of this successor
            if r_R:
                if nd.parent == 0:
                    root_pad[nd.slot] += r_R
                else:
                    state.cores[nd.parent] = _pad_axis(state.cores[nd.parent], nd.slot, r_R)
        # Step 1 revisited: project onto the updated cores of the layer
        for nd in tree.layer_nodes(layer):
            C = mode_product_t(C, axes.index(nd.id), new_bases[nd.id][0])
    # eq. incremental_root_concatenate with the root padded first (R8)
    root = _pad_axis(_pad_axis(state.root, 0, root_pad[0]), 1, root_pad[1])
    state.root = np.concatenate([root, C], axis=2)
    state.n_items += C.shape[-1]
    return UpdateInfo(False, eps_proj, eps_des, ranks_before, state.ranks())


# ---------------------------------------------------------------------------
# Reconstruction root-to-leaves (eq. htucker_reconstruction, R11)
# ---------------------------------------------------------------------------

def decode(state: BHTState, Z: np.ndarray) -> np.ndarray:
    """Root-to-leaves expansion (eq. htucker_reconstruction) of latent items Z, item-major
    [N, r_11, r_12], into [N, n_1..n_d]: every node's core contracted in, layer by layer."""
    tree = state.tree
    C = np.moveaxis(np.asarray(Z, dtype=np.float64), 0, -1)      # [r_11, r_12, N]
    tags = list(tree.nodes[0].children)          # axis -> node id still to expand
    for layer in range(1, tree.p + 1):
        for nd in tree.layer_nodes(layer):
            ax = tags.index(nd.id)
            G = state.cores[nd.id]
            if nd.is_leaf:
                C = np.moveaxis(np.tensordot(C, G, axes=([ax], [1])), -1, ax)
                tags[ax] = ("mode", nd.mode)
            else:
                out = np.tensordot(C, G, axes=([ax], [2]))       # children axes appended last
                C = np.moveaxis(out, [-2, -1], [ax, ax + 1])
                tags[ax:ax + 1] = list(nd.children)
    assert tags == [("mode", m) for m in range(tree.d)]
    return np.moveaxis(C, -1, 0)


def reconstruct(state: BHTState, first: int = 0, count: int = None) -> np.ndarray:
    """Decode items first..first+count-1 of the accumulation, item-major [count, n_1..n_d]."""
    if count is None:
        count = state.n_items - first
    return decode(state, np.moveaxis(state.root[:, :, first:first + count], -1, 0))


def relative_test_error(state: BHTState, X: np.ndarray, per_item: bool = False):
    """eq. generalization_performance: the mean over the items X_i (which need not be in the
    accumulation) of ||X_i - decode(project(X_i))|| / ||X_i||; an all-zero item counts 0."""
    X = np.asarray(X, dtype=np.float64)
    E = X - decode(state, project(state, X))
    errs = np.array([np.linalg.norm(E[i]) / np.linalg.norm(X[i]) if np.any(X[i]) else 0.0
                     for i in range(X.shape[0])])
    return (float(errs.mean()), errs) if per_item else float(errs.mean())


def reduction_ratio(state: BHTState) -> float:
    """eq. reduction_ratio: elements of one item over elements of its latent representation (r_11 r_12)."""
    r = state.ranks()
    return int(np.prod(state.tree.dims)) / (r[1] * r[2])


def normalize(Y: np.ndarray, kind: str, groups: int = None):
    """Normalisation of the scientific-data experiments (Sec. 5.2), each group of consecutive elements on
    its own (default one group per item): maxabs Y / max|Y|, unitvec Y / ||Y||, zscore (Y - mean) / std
    with the population standard deviation; a zero or non-finite scale is replaced by 1. Returns the
    normalised float64 array and the (shift, scale) rows."""
    Y = np.asarray(Y, dtype=np.float64)
    groups = Y.shape[0] if groups is None else groups
    G = Y.reshape(groups, -1)
    shift = np.zeros(groups)
    if kind == "maxabs":
        scale = np.abs(G).max(axis=1)
    elif kind == "unitvec":
        scale = np.sqrt((G * G).sum(axis=1))
    elif kind == "zscore":
        shift = G.mean(axis=1)
        scale = np.sqrt(((G - shift[:, None]) ** 2).mean(axis=1))
    elif kind == "none":
        scale = np.ones(groups)
    else:
        raise ValueError(kind)
    scale = np.where((scale > 0) & np.isfinite(scale), scale, 1.0)
    return ((G - shift[:, None]) / scale[:, None]).reshape(Y.shape), np.column_stack([shift, scale])


def compression_ratio(state: BHTState, n_items_elements: int = None) -> float:
    """eq. compression_ratio: elements of the accumulation / elements of all HT cores."""
    if n_items_elements is None:
        n_items_elements = state.n_items * int(np.prod(state.tree.dims))
    return n_items_elements / state.num_elements()

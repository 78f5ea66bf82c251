"""Full-rank certificate (bht_eig_min_above) and the identity bases BHT-l2r gives certified nodes.

The tail rule of eq. ht_leaf_svd keeps all n directions of a node exactly when the smallest eigenvalue
of its Gram matrix exceeds eps_nw^2. The certificate is a Cholesky factorisation of G - (tau + delta) I
in FP64, delta = 2 (n + 4) 2^-53 trace(G); it must say yes whenever lambda_min exceeds tau by more than
delta and may only say yes when lambda_min > tau.

* matrices with a known spectrum (Q diag(lam) Q^T): tau just below and just above lambda_min, at tile
  multiples and ragged sizes, the n = 343 of the 24^5 sensor stream's largest interior node, 600;
* rank-deficient Gram matrices, a non-finite entry, argument errors;
* BHT-l2r on a tensor of known multilinear ranks whose interior nodes are full rank: their cores are the
  identity, the reconstruction and the ranks are the oracle's; an update that grows a leaf pads the
  parent, which is then no longer the identity and expands like any other node (both precisions).
"""
import ctypes

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


def _spd(n, lam, seed):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.normal(size=(n, n)))[0]
    G = (Q * lam) @ Q.T
    return 0.5 * (G + G.T)


@pytest.mark.parametrize("n", [1, 7, 16, 17, 49, 100, 343, 600])
def test_certificate_against_known_spectrum(B, n):
    lam = np.logspace(0, 2, n)[::-1].copy()
    G = _spd(n, lam, n)
    lmin = np.linalg.eigvalsh(G)[0]  # the spectrum of the rounded matrix
    Gd = torch.from_numpy(G).cuda()
    before = Gd.clone()
    assert B.bht_eig_min_above(Gd, lmin * (1 - 1e-6))
    assert not B.bht_eig_min_above(Gd, lmin * (1 + 1e-6))
    assert not B.bht_eig_min_above(Gd, 10.0 * lam[0])
    assert torch.equal(Gd, before)  # G is not written


@pytest.mark.parametrize("n", [2, 16, 33, 343])
def test_certificate_refuses_singular_and_non_finite(B, n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, n // 2))
    G = X @ X.T  # rank n // 2: lambda_min = 0
    assert not B.bht_eig_min_above(torch.from_numpy(G).cuda(), 0.0)
    H = _spd(n, np.linspace(1.0, 2.0, n), n)
    H[n - 1, n // 2] = H[n // 2, n - 1] = np.nan
    assert not B.bht_eig_min_above(torch.from_numpy(H).cuda(), 0.0)
    assert not B.bht_eig_min_above(torch.zeros((n, n), dtype=torch.float64, device="cuda"), 0.0)


def test_certificate_arguments(B):
    G = torch.eye(4, dtype=torch.float64, device="cuda")
    v = ctypes.c_int32(7)
    lib = B._lib
    assert lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), 4, -1.0, ctypes.byref(v), None) == B.BHT_EINVAL
    assert lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), 4, float("inf"), ctypes.byref(v), None) == B.BHT_EINVAL
    assert lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), 0, 0.0, ctypes.byref(v), None) == B.BHT_EINVAL
    assert lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), 4097, 0.0, ctypes.byref(v), None) == B.BHT_ECAPACITY
    host = np.eye(4)
    assert lib.bht_eig_min_above(ctypes.c_void_p(host.ctypes.data), 4, 0.0, ctypes.byref(v), None) == B.BHT_EINVAL
    assert lib.bht_eig_min_above(ctypes.c_void_p(G.data_ptr()), 4, 0.5, ctypes.byref(v), None) == B.BHT_OK
    assert v.value == 1


def _known_ranks(rng, N, ranks, bases):
    core = rng.normal(size=(N,) + tuple(b.shape[1] for b in bases))
    for m, r in enumerate(ranks):
        idx = [slice(None)] * core.ndim
        idx[m + 1] = slice(r, None)
        core[tuple(idx)] = 0.0
    return np.einsum("nabcd,ia,jb,kc,ld->nijkl", core, *bases)


def _core(B, st, node, shape):
    n = int(np.prod(shape))
    out = np.empty(n)
    numel = ctypes.c_int64()
    B._check(B._lib.bht_get_core(st, node, out.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(numel)),
             "bht_get_core")
    assert numel.value == n
    return out.reshape(shape)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_identity_bases_then_growth(B, precision):
    rng = np.random.default_rng(5)
    dims = (6, 7, 5, 6)
    bases = [np.linalg.qr(rng.normal(size=(n, 3)))[0] for n in dims]
    Y1 = _known_ranks(rng, 24, (2, 2, 2, 2), bases)  # interior nodes: 2 x 2 = 4 rows, all kept
    Y2 = _known_ranks(rng, 24, (3, 2, 2, 2), bases)  # leaf of mode 0 grows to 3
    eps = 1e-6
    tree = B.bht_tree_create_balanced(dims)
    dt = torch.float64 if precision == "fp64" else torch.float32
    st = B.bht_l2r(tree, torch.from_numpy(Y1).to(dt).cuda(), eps, precision=precision)
    ost = O.bht_l2r(Y1, eps)
    g = B.bht_get_ranks(st)
    assert g[1:] == ost.ranks()[1:]
    t = O.dimension_tree(dims)
    interior = [nd for nd in t.nodes if not nd.is_leaf and nd.id > 0]
    assert interior
    for nd in interior:
        ra, rb = g[nd.children[0]], g[nd.children[1]]
        assert g[nd.id] == ra * rb
        assert np.array_equal(_core(B, st, nd.id, (ra, rb, ra * rb)).reshape(ra * rb, ra * rb), np.eye(ra * rb))
    tol = 1e-10 if precision == "fp64" else 2e-5
    Yg = B.ht_reconstruct(st, 0, 24, dtype="float64").cpu().numpy()
    assert np.linalg.norm(Yg - O.reconstruct(ost)) <= tol * np.linalg.norm(Y1)

    info = B.htrise_update(st, torch.from_numpy(Y2).to(dt).cuda(), eps, precision=precision)
    oinfo = O.htrise_update(ost, Y2, eps)
    assert info.skipped == oinfo.skipped is False
    g = B.bht_get_ranks(st)
    assert g[1:] == ost.ranks()[1:]
    leaf0 = t.leaf_of_mode[0]
    assert g[leaf0] == 3
    par = next(nd for nd in interior if leaf0 in nd.children)
    ra, rb = g[par.children[0]], g[par.children[1]]
    assert g[par.id] == ra * rb == 6
    Up = _core(B, st, par.id, (ra, rb, g[par.id])).reshape(ra * rb, g[par.id])
    assert not np.array_equal(Up, np.eye(ra * rb))  # padded, then expanded: no longer the identity
    assert np.abs(Up.T @ Up - np.eye(g[par.id])).max() < 1e-10
    Yg = B.ht_reconstruct(st, 0, 48, dtype="float64").cpu().numpy()
    Yall = np.concatenate([Y1, Y2])
    assert np.linalg.norm(Yg - O.reconstruct(ost)) <= tol * np.linalg.norm(Yall)
    # a third batch in the old span: the state after growth still skips
    Y3 = _known_ranks(rng, 8, (3, 2, 2, 2), bases)
    info = B.htrise_update(st, torch.from_numpy(Y3).to(dt).cuda(), eps, precision=precision)
    assert info.skipped
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)

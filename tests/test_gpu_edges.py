"""Degenerate and boundary cases of the compression calls, through the C ABI.

* an all-zero batch: every node keeps rank 1 (the tail rule's minimum), the reconstruction is exactly
  zero, a later all-zero increment skips, and a later non-zero increment expands within the bound;
* a batch of separable (rank-one) items: every rank is 1 and the reconstruction is exact;
* the same increment twice: the second update skips and changes no rank;
* a node beyond the eigensolver's 4096 rows: BHT_ECAPACITY before any work, the library still usable;
* a leaf of 3000 rows, too large for the shared-memory tridiagonalisation: the global-memory kernel,
  checked against the oracle.
"""
import numpy as np
import pytest

import bht_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


def dev(Y):
    return torch.from_numpy(np.ascontiguousarray(Y)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_all_zero_batches(B, precision):
    dims = (6, 7, 5)
    tree = B.bht_tree_create_balanced(dims)
    st = B.bht_l2r(tree, dev(np.zeros((4,) + dims, np.float32)), 0.1, precision=precision)
    assert B.bht_get_ranks(st) == [4, 1, 1, 1, 1]
    assert float(B.ht_reconstruct(st, 0, 4, dtype="float64").abs().max()) == 0.0
    info = B.htrise_update(st, dev(np.zeros((3,) + dims, np.float32)), 0.1, precision=precision)
    assert info.skipped and info.eps_proj == 0.0 and B.bht_get_ranks(st)[0] == 7
    Y = np.random.default_rng(1).normal(size=(3,) + dims).astype(np.float32)
    info = B.htrise_update(st, dev(Y), 0.1, precision=precision)
    assert not info.skipped
    rec = B.ht_reconstruct(st, 7, 3, dtype="float64").cpu().numpy()
    assert np.linalg.norm(rec - Y) <= 0.1 * np.linalg.norm(Y) * (1 + 1e-6)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_rank_one_items_are_exact(B):
    rng = np.random.default_rng(2)
    dims = (9, 8, 7, 6)
    a, b, c, d = (rng.normal(size=n) for n in dims)
    scale = rng.normal(size=5)
    Y = np.einsum("n,i,j,k,l->nijkl", scale, a, b, c, d)
    tree = B.bht_tree_create_balanced(dims)
    st = B.bht_l2r(tree, dev(Y), 1e-6, precision="fp64")
    assert B.bht_get_ranks(st)[1:] == [1] * 6
    assert rel(B.ht_reconstruct(st, 0, 5, dtype="float64").cpu().numpy(), Y) < 1e-12
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_repeated_increment_skips(B, precision):
    Y = S.spectral_field(4, 0, 16, n=32)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, dev(Y), 1e-2, precision=precision)
    before = B.bht_get_ranks(st)
    info = B.htrise_update(st, dev(Y), 1e-2, precision=precision)
    assert info.skipped and info.eps_proj <= info.eps_des
    after = B.bht_get_ranks(st)
    assert after[0] == 32 and after[1:] == before[1:]
    # the copy reconstructs as the original does
    a = B.ht_reconstruct(st, 0, 16, dtype="float64").cpu().numpy()
    b = B.ht_reconstruct(st, 16, 16, dtype="float64").cpu().numpy()
    assert rel(b, a) < (1e-12 if precision == "fp64" else 1e-5)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_node_beyond_the_eigensolver_limit(B):
    # full-rank 70 x 70 leaves make node {1,2} a 4900-row unfolding
    Y = np.random.default_rng(3).normal(size=(3, 70, 70, 3)).astype(np.float32)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    with pytest.raises(B.BHTError) as err:
        B.bht_l2r(tree, dev(Y), 1e-3)
    assert err.value.status == B.BHT_ECAPACITY
    B.bht_tree_destroy(tree)
    tree = B.bht_tree_create_balanced((7, 9))          # still usable
    st = B.bht_l2r(tree, dev(np.ones((2, 7, 9), np.float32)), 0.1)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_large_leaf_global_memory_tridiagonalisation(B):
    rng = np.random.default_rng(4)
    Y = rng.normal(size=(2, 3000, 3))
    Y[:, :, 1] += np.cumsum(rng.normal(size=(2, 3000)), axis=1) * 0.01
    eps = 1e-3
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, dev(Y), eps, precision="fp64")
    ost = O.bht_l2r(Y, eps)
    assert B.bht_get_ranks(st)[1:] == ost.ranks()[1:]
    g = B.ht_reconstruct(st, 0, 2, dtype="float64").cpu().numpy()
    assert rel(g, O.reconstruct(ost)) < 1e-9
    assert np.linalg.norm(g - Y) <= eps * np.linalg.norm(Y) * (1 + 1e-9)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)

"""Decoding of latent items (eq. htucker_reconstruction) and the relative test error of unseen items
(encode with Step 1 of Algorithm 2, then decode), GPU path against the FP64 oracle.

Both sides run on the same cores: the GPU's cores are copied into an oracle state, so the comparison
is element by element. Tolerances: FP64 path 1e-12 relative (rounding of a few contractions of length
<= 4096). Mixed path 5e-5: its mode products run on the tensor cores in split TF32, about 2^-20 relative
per product, so an output summed over K terms of an orthonormal basis is off by up to about
2^-20 sqrt(K) of its scale, 3e-5 for the K ~ 1000 of a transfer node. A relative test error inherits
that as an absolute difference (each item's reconstruction is off by that fraction of the item).
"""
import numpy as np
import pytest

import bht_synth as S
import oracle as O
import oracle.bht_oracle as OB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 5e-5}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(Y):
    return torch.from_numpy(np.ascontiguousarray(Y)).cuda()


def oracle_copy(B, st, dims):
    """An oracle state holding the GPU's cores and root (same layouts: leaf [n, r], transfer [r_a, r_b, r])."""
    tree = OB.dimension_tree(dims)
    ranks = B.bht_get_ranks(st)
    cores = {}
    for nd in tree.nodes[1:]:
        c = B.bht_get_core(st, nd.id)
        if nd.is_leaf:
            cores[nd.id] = c.reshape(dims[nd.mode], ranks[nd.id])
        else:
            a, b = nd.children
            cores[nd.id] = c.reshape(ranks[a], ranks[b], ranks[nd.id])
    root = np.moveaxis(B.bht_get_root(st, 0, ranks[0]), 0, -1)
    return OB.BHTState(tree=tree, eps_rel=0.0, cores=cores, root=root, n_items=ranks[0])


def stream_state(B, Y, inc, eps, precision):
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, to_dev(Y[:inc]), eps, precision=precision)
    for k in range(inc, Y.shape[0], inc):
        B.htrise_update(st, to_dev(Y[k:k + inc]), eps, precision=precision)
    return tree, st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dims,items,inc,eps", [
    ((7, 9), 6, 3, 0.05),
    ((5, 6, 7), 9, 3, 0.1),
    ((3, 4, 5, 3, 4), 12, 4, 0.02),
    ((32, 32, 32), 24, 8, 1e-2),
])
def test_decode_matches_oracle_on_the_same_cores(B, precision, dims, items, inc, eps):
    rng = np.random.default_rng(len(dims) * 100 + items)
    Y = rng.normal(size=(items,) + dims) + np.cumsum(rng.normal(size=(items,) + dims), axis=1)
    if len(dims) == 3 and dims[0] == 32:
        Y = S.spectral_field(5, 0, items, n=32)
    tree, st = stream_state(B, Y, inc, eps, precision)
    ost = oracle_copy(B, st, dims)
    r = B.bht_get_ranks(st)
    for N in (1, 5, 37):                                         # N = 37: several tiles and a ragged tail
        Z = rng.normal(size=(N, r[1], r[2]))
        want = O.decode(ost, Z)
        got_h = B.ht_decode(st, Z, dtype="float64").cpu().numpy()            # host latent
        got_d = B.ht_decode(st, to_dev(Z), dtype="float64").cpu().numpy()    # device latent
        assert rel(got_h, want) <= TOL[precision]
        assert np.array_equal(got_h, got_d)
        got32 = B.ht_decode(st, to_dev(Z), dtype="float32").cpu().numpy()
        assert rel(got32, want) <= max(TOL[precision], 2 ** -23)
        host_out = np.empty((N,) + dims, dtype=np.float64)                     # host output buffer
        B.ht_decode(st, Z, out=host_out)
        assert np.array_equal(host_out, got_h)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_reconstruct_is_decode_of_the_root(B, precision):
    Y = S.gaussian_bumps(1, 0, 24)
    tree, st = stream_state(B, Y, 8, 1e-3, precision)
    for first, count in ((0, 24), (5, 1), (9, 13)):
        Z = B.bht_get_root(st, first, count)
        a = B.ht_reconstruct(st, first, count, dtype="float64").cpu().numpy()
        b = B.ht_decode(st, Z, dtype="float64").cpu().numpy()
        assert np.array_equal(a, b)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_relative_test_error_matches_oracle(B, precision):
    # the spectral stream at 32^3: three increments accumulated, then items of later snapshots that the
    # cores never saw; the RTE is the mean of the per-item relative errors (eq. generalization_performance)
    Y = S.spectral_field(7, 0, 24, n=32)
    eps = 1e-2
    tree, st = stream_state(B, Y, 8, eps, precision)
    ost = oracle_copy(B, st, Y.shape[1:])
    X = S.spectral_field(7, 40, 6, n=32)
    got, gerr = B.relative_test_error(st, to_dev(X), per_item=True)
    want, werr = O.relative_test_error(ost, X, per_item=True)
    assert np.abs(gerr - werr).max() <= TOL[precision] * 10 + 1e-14
    assert abs(got - want) <= TOL[precision] * 10 + 1e-14
    assert got > 0.0
    got_h = B.relative_test_error(st, X)                       # host items: the same numbers
    assert abs(got_h - got) <= 1e-15 + TOL[precision] * 1e-3
    # encoded latents agree element by element with the oracle's projection on the same cores
    Zg = B.ht_encode(st, to_dev(X))
    Zo = O.project(ost, X)
    assert rel(Zg, Zo) <= TOL[precision]
    # the last stored increment: the projection is the best in the frames' span, so its aggregate error
    # is at most the stored approximation's, which meets the per-increment bound
    last = Y[16:24]
    _, e = B.relative_test_error(st, to_dev(last), per_item=True)
    nrm = np.linalg.norm(last.reshape(8, -1).astype(np.float64), axis=1)
    assert np.sqrt(np.sum((e * nrm) ** 2)) <= eps * np.linalg.norm(nrm) * (1 + 1e-4)
    # items of the represented subspace come back unchanged; an all-zero item counts 0
    r = B.bht_get_ranks(st)
    Xs = O.decode(ost, np.random.default_rng(8).normal(size=(3, r[1], r[2])))
    assert B.relative_test_error(st, to_dev(Xs)) <= TOL[precision] * 10
    Xz = np.concatenate([X[:2], np.zeros_like(X[:1])])
    assert abs(B.relative_test_error(st, to_dev(Xz)) - np.mean(gerr[:2]) * 2 / 3) <= TOL[precision] * 10
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_relative_test_error_full_size_sampled(B):
    """The spectral stream at its full 64^3 grid, increments of 32, mixed path; the oracle decodes the
    sampled held-out items on the GPU's cores."""
    Y = S.spectral_field(0, 0, 96, n=64)
    tree, st = stream_state(B, Y, 32, 1e-2, "mixed")
    ost = oracle_copy(B, st, Y.shape[1:])
    X = S.spectral_field(0, 200, 4, n=64)
    got = B.relative_test_error(st, to_dev(X))
    assert abs(got - O.relative_test_error(ost, X)) <= 1e-4
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_empty_batches(B):
    Y = S.spectral_field(2, 0, 4, n=16)
    tree, st = stream_state(B, Y, 4, 1e-2, "fp64")
    r = B.bht_get_ranks(st)
    Z = B.ht_encode(st, np.empty((0, 16, 16, 16), dtype=np.float32))
    assert Z.shape == (0, r[1], r[2])
    D = B.ht_decode(st, np.empty((0, r[1], r[2])))
    assert D.shape == (0, 16, 16, 16)
    with pytest.raises(TypeError):
        B.ht_decode(st, np.empty((2, r[1], r[2]), dtype=np.float32))
    with pytest.raises(ValueError):
        B.ht_decode(st, np.empty((2, r[1] + 1, r[2])))
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)

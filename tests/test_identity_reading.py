"""The reading that a node whose truncation keeps every direction takes the identity as its basis.

The truncated SVD of eq. ht_leaf_svd gives, for a node that keeps all of its rows' directions, one
orthonormal basis of the whole space among many; every such basis has U U^T = I. Replacing it by the
identity (the GPU path's choice for a node a Cholesky certificate shows to be full rank) must leave every
projection and reconstruction as it was: the items re-encoded on the modified cores decode to the oracle's
reconstruction. Checked with the oracle alone, on the Chebyshev sensor stream at 12^4 (every interior node
full rank at eps = 1e-2) and on a tensor of known multilinear ranks.
"""
import copy

import numpy as np

import bht_synth as S
import oracle as O


def _identity_cores(st):
    """A copy of the state with every full-rank interior core replaced by the identity; the ids replaced."""
    out = copy.deepcopy(st)
    replaced = []
    for nd in st.tree.nodes:
        if nd.id == 0 or nd.is_leaf:
            continue
        G = st.cores[nd.id]
        ra, rb, r = G.shape
        if r == ra * rb:
            out.cores[nd.id] = np.eye(r).reshape(ra, rb, r)
            replaced.append(nd.id)
    return out, replaced


def _check(Y, eps):
    st = O.bht_l2r(Y, eps)
    st_id, replaced = _identity_cores(st)
    assert replaced, "no full-rank interior node in this case"
    Yh = O.reconstruct(st)
    Yi = O.decode(st_id, O.project(st_id, Y))
    assert np.linalg.norm(Yi - Yh) <= 1e-12 * np.linalg.norm(Y)
    # and the bound of eq. ht_leaf_svd still holds for the modified cores (the same projection)
    assert np.linalg.norm(Yi - Y) <= eps * np.linalg.norm(Y) * (1 + 1e-9)
    return st, replaced


def test_identity_basis_for_full_rank_nodes_sensor():
    Y = S.chebyshev_sensor(0, 0, 8, n=12, d=4)
    st, replaced = _check(Y, 1e-2)
    # both interior nodes of the balanced 4-mode tree are full rank (7 x 7 = 49 rows, rank 49)
    assert len(replaced) == 2


def test_identity_basis_for_full_rank_nodes_known_ranks():
    rng = np.random.default_rng(5)
    dims = (6, 7, 5, 6)
    bases = [np.linalg.qr(rng.normal(size=(n, 2)))[0] for n in dims]
    core = rng.normal(size=(16, 2, 2, 2, 2))
    Y = np.einsum("nabcd,ia,jb,kc,ld->nijkl", core, *bases)
    _check(Y, 1e-6)


def test_a_rotated_basis_is_not_the_identity_but_gives_the_same_items():
    """Any orthonormal basis of the full space works, not only the one the SVD returns: a random rotation
    of a full-rank core re-encodes to the same items (the check above does not depend on the identity)."""
    Y = S.chebyshev_sensor(1, 0, 6, n=12, d=4)
    st = O.bht_l2r(Y, 1e-2)
    rng = np.random.default_rng(0)
    rot = copy.deepcopy(st)
    for nd in st.tree.nodes:
        if nd.id == 0 or nd.is_leaf:
            continue
        G = st.cores[nd.id]
        ra, rb, r = G.shape
        if r == ra * rb:
            Q = np.linalg.qr(rng.normal(size=(r, r)))[0]
            rot.cores[nd.id] = (G.reshape(r, r) @ Q).reshape(ra, rb, r)
    Yr = O.decode(rot, O.project(rot, Y))
    assert np.linalg.norm(Yr - O.reconstruct(st)) <= 1e-12 * np.linalg.norm(Y)


def test_the_check_sees_a_basis_that_does_not_span_the_kept_space():
    """The same re-encoding with a leaf's basis (rank 7 of 12 rows) replaced by the first columns of the
    identity changes the items: the check above is not blind to a wrong basis."""
    Y = S.chebyshev_sensor(0, 0, 8, n=12, d=4)
    st = O.bht_l2r(Y, 1e-2)
    bad = copy.deepcopy(st)
    leaf = next(nd for nd in st.tree.nodes if nd.is_leaf)
    n, r = st.cores[leaf.id].shape
    assert r < n
    bad.cores[leaf.id] = np.eye(n)[:, :r]
    Yb = O.decode(bad, O.project(bad, Y))
    assert np.linalg.norm(Yb - O.reconstruct(st)) > 1e-3 * np.linalg.norm(Y)

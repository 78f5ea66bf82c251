"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks reuses the oracle's own formulas: expected values come
from closed forms, textbook special cases (LAPACK SVD / symmetric eigen),
exact constructions with known ranks, explicit loops on tiny inputs, and the
theorems of Appendix A.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import bht_synth as S
import oracle as O
import oracle.bht_oracle as OB

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers independent of the oracle
# ---------------------------------------------------------------------------

def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def rand_orth(rng, rows, cols):
    Q, _ = np.linalg.qr(rng.normal(size=(rows, cols)))
    return Q


def brute_rank(sig2, thr2, rmin):
    """Smallest r >= rmin whose discarded energy is <= thr2, by trying every r."""
    for r in range(rmin, len(sig2) + 1):
        if sum(sig2[r:]) <= thr2:
            return r
    return len(sig2)


def principal_sin(U, V):
    """Largest sine of the principal angles between span(U) and span(V)."""
    return float(np.linalg.norm(V - U @ (U.T @ V), 2))


def tree_d5_exact(rng, dims, ranks, N):
    """Random batch-HT tensor on the 5-mode tree of Fig. 2 (left), written as one einsum.

    ranks: dict with leaf ranks r0..r4, transfer ranks r01, r012, r34.
    """
    n0, n1, n2, n3, n4 = dims
    U = [rand_orth(rng, dims[i], ranks[f"r{i}"]) for i in range(5)]
    G01 = rand_orth(rng, ranks["r0"] * ranks["r1"], ranks["r01"]).reshape(ranks["r0"], ranks["r1"], ranks["r01"])
    G012 = rand_orth(rng, ranks["r01"] * ranks["r2"], ranks["r012"]).reshape(ranks["r01"], ranks["r2"], ranks["r012"])
    G34 = rand_orth(rng, ranks["r3"] * ranks["r4"], ranks["r34"]).reshape(ranks["r3"], ranks["r4"], ranks["r34"])
    root = rng.normal(size=(ranks["r012"], ranks["r34"], N))
    Y = np.einsum("abn,xyc,cza,pqb,ix,jy,kz,lp,mq->nijklm",
                  root, G01, G012, G34, U[0], U[1], U[2], U[3], U[4], optimize=True)
    return Y, U


# ---------------------------------------------------------------------------
# Dimension tree (Section 2.3, Fig. 2)
# ---------------------------------------------------------------------------

def test_tree_matches_fig2_left():
    lines = [l.strip() for l in open(os.path.join(GOLDEN, "tree_fig2_left.txt")) if l.strip() and not l.startswith("#")]
    expect = [[tuple(int(x) - 1 for x in grp.split(",")) for grp in line.split("|")] for line in lines]
    t = O.dimension_tree((4, 5, 6, 7, 8))
    got = [[nd.modes for nd in t.layer_nodes(l)] for l in range(t.p + 1)]
    assert got == expect


@pytest.mark.parametrize("d", range(2, 17))
def test_tree_depth_and_leaf_layers(d):
    t = O.dimension_tree([3] * d)
    assert t.p == math.ceil(math.log2(d))                    # Section 2.3
    assert len(t.nodes) == 2 * d - 1                          # 2d - 1 nodes
    leaves = [nd for nd in t.nodes if nd.is_leaf]
    assert sorted(nd.mode for nd in leaves) == list(range(d))
    assert {nd.layer for nd in leaves} <= {t.p, t.p - 1}      # balanced: leaves on p and p-1
    for nd in t.nodes[1:]:                                    # successors ordered by position
        par = t.nodes[nd.parent]
        assert par.children[nd.slot] == nd.id
        assert par.modes == t.nodes[par.children[0]].modes + t.nodes[par.children[1]].modes


# ---------------------------------------------------------------------------
# Truncation rule (eq. ht_leaf_svd)
# ---------------------------------------------------------------------------

def test_truncation_rank_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(300):
        k = int(rng.integers(1, 12))
        s2 = np.sort(rng.exponential(size=k) * (rng.random(k) < 0.8))[::-1]
        thr = float(rng.uniform(0, 1.2)) * s2.sum()
        for rmin in (0, 1):
            assert O.bht_oracle.truncation_rank(s2, thr, rmin) == brute_rank(list(s2), thr, rmin)
    # equality is allowed: a tail exactly at the threshold is discarded
    assert O.bht_oracle.truncation_rank(np.array([4.0, 1.0]), 1.0, 1) == 1


# ---------------------------------------------------------------------------
# Special cases that reduce to textbook routines
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eps", [0.3, 0.05, 1e-3])
def test_d2_single_item_is_truncated_svd(eps):
    """d = 2, N = 1: BHT-l2r is the truncated SVD of a matrix (Eckart-Young)."""
    rng = np.random.default_rng(2)
    A = rng.normal(size=(9, 7)) @ np.diag(0.5 ** np.arange(7)) @ rng.normal(size=(7, 7))
    U, s, Vt = scipy.linalg.svd(A, lapack_driver="gesvd")
    thr2 = (eps * np.linalg.norm(A)) ** 2 / 2.0     # eps_nw^2 with 2d - 2 = 2
    r = brute_rank(list(s * s), thr2, 1)
    best = (U[:, :r] * s[:r]) @ Vt[:r]
    st = O.bht_l2r(A[None], eps)
    assert st.ranks()[1:] == [r, r]
    assert rel(O.reconstruct(st)[0], best) < 1e-12
    G0 = st.root[:, :, 0]
    assert np.allclose(np.abs(G0), np.diag(s[:r]), atol=1e-12 * s[0])


def test_d2_batch_is_truncated_hosvd():
    """d = 2, batch N: leaves are the truncated HOSVD bases of the n1 x n2 x N tensor on modes 1, 2."""
    rng = np.random.default_rng(3)
    n1, n2, N, eps = 8, 6, 5, 0.05
    Y = np.einsum("ia,jb,abn->nij", rng.normal(size=(n1, 4)), rng.normal(size=(n2, 3)),
                  rng.normal(size=(4, 3, N))) + 0.02 * rng.normal(size=(N, n1, n2))
    # mode Grams by explicit loops, eigen by LAPACK syevd
    G1 = np.zeros((n1, n1)); G2 = np.zeros((n2, n2))
    for n in range(N):
        for i in range(n1):
            for j in range(n2):
                G1[i] += Y[n, i, j] * Y[n, :, j]
                G2[j] += Y[n, i, j] * Y[n, i, :]
    thr2 = (eps * np.linalg.norm(Y)) ** 2 / 2.0
    P = []
    for G in (G1, G2):
        w, V = np.linalg.eigh(G)
        w, V = w[::-1], V[:, ::-1]
        r = brute_rank(list(np.clip(w, 0, None)), thr2, 1)
        P.append(V[:, :r] @ V[:, :r].T)
    expect = np.einsum("ia,naj,jb->nib", P[0], Y, P[1])
    st = O.bht_l2r(Y, eps)
    assert rel(O.reconstruct(st), expect) < 1e-10
    assert rel(O.reconstruct(st), Y) <= eps


# ---------------------------------------------------------------------------
# Brute force on a tiny 3-mode batch: every node rank from explicit loops
# ---------------------------------------------------------------------------

def test_tiny_brute_force_ranks_and_root():
    rng = np.random.default_rng(4)
    N, n1, n2, n3, eps = 2, 3, 4, 5, 0.2
    Y = rng.normal(size=(N, n1, n2, n3))
    st = O.bht_l2r(Y, eps)
    t = st.tree
    thr2 = (eps * np.linalg.norm(Y)) ** 2 / 4.0            # 2d - 2 = 4 for d = 3
    leaf = {nd.mode: nd.id for nd in t.nodes if nd.is_leaf}
    n12 = t.nodes[0].children[0]

    def rank_of(M):
        G = np.zeros((M.shape[0], M.shape[0]))
        for c in range(M.shape[1]):
            G += np.outer(M[:, c], M[:, c])
        w = np.clip(np.linalg.eigvalsh(G)[::-1], 0, None)
        return brute_rank(list(w), thr2, 1)

    # layer 2 leaves (modes 1, 2) from Y itself
    M1 = np.array([[Y[n, i, j, k] for n in range(N) for j in range(n2) for k in range(n3)] for i in range(n1)])
    M2 = np.array([[Y[n, i, j, k] for n in range(N) for i in range(n1) for k in range(n3)] for j in range(n2)])
    assert st.rank(leaf[0]) == rank_of(M1)
    assert st.rank(leaf[1]) == rank_of(M2)
    U1, U2 = st.cores[leaf[0]], st.cores[leaf[1]]
    r1, r2 = U1.shape[1], U2.shape[1]
    # layer-1 intermediate C1[n, a*r2+b, k] by loops (C-order merge, reading R4)
    C1 = np.zeros((N, r1 * r2, n3))
    for n in range(N):
        for a in range(r1):
            for b in range(r2):
                for k in range(n3):
                    C1[n, a * r2 + b, k] = sum(U1[i, a] * U2[j, b] * Y[n, i, j, k]
                                               for i in range(n1) for j in range(n2))
    M12 = np.array([[C1[n, q, k] for n in range(N) for k in range(n3)] for q in range(r1 * r2)])
    M3 = np.array([[C1[n, q, k] for n in range(N) for q in range(r1 * r2)] for k in range(n3)])
    assert st.rank(n12) == rank_of(M12)
    assert st.rank(leaf[2]) == rank_of(M3)
    # root = C1 projected on both layer-1 bases
    U12 = st.basis(n12)
    U3 = st.cores[leaf[2]]
    root = np.einsum("nqk,qa,kb->abn", C1, U12, U3)
    assert rel(st.root, root) < 1e-12


# ---------------------------------------------------------------------------
# Exact recovery of tensors built with known HT ranks
# ---------------------------------------------------------------------------

RANKS_D5 = dict(r0=2, r1=3, r2=2, r3=3, r4=2, r01=4, r012=5, r34=3)


def test_exact_recovery_known_ranks_d5():
    rng = np.random.default_rng(5)
    dims = (4, 5, 3, 6, 7)
    Y, U = tree_d5_exact(rng, dims, RANKS_D5, N=40)
    st = O.bht_l2r(Y, 1e-10)
    t = st.tree
    names = {t.nodes[0].children[0]: "r012", t.nodes[0].children[1]: "r34"}
    for nd in t.nodes[1:]:
        if nd.is_leaf:
            names[nd.id] = f"r{nd.mode}"
        elif nd.modes == (0, 1):
            names[nd.id] = "r01"
    got = {names[nd.id]: st.rank(nd.id) for nd in t.nodes[1:]}
    assert got == RANKS_D5
    assert rel(O.reconstruct(st), Y) < 1e-12
    for nd in t.nodes[1:]:
        if nd.is_leaf:
            assert principal_sin(st.cores[nd.id], U[nd.mode]) < 1e-10


# ---------------------------------------------------------------------------
# Error bound (Corollary bht_leaves_to_root, Problem 1) and Claim (orthogonal reconstructions)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(6, 7), (5, 4, 6), (3, 4, 5, 3), (3, 3, 4, 3, 3), (2, 3, 2, 3, 2, 3)])
@pytest.mark.parametrize("eps", [0.3, 0.1, 0.01])
def test_bht_error_bound_and_norm_identity(dims, eps):
    rng = np.random.default_rng(hash((dims, eps)) % 2 ** 32)
    base = rng.normal(size=(6,) + dims)
    Y = base + 0.3 * np.roll(base, 1, axis=0) ** 2
    st = O.bht_l2r(Y, eps)
    Yh = O.reconstruct(st)
    err = np.linalg.norm(Y - Yh)
    assert err <= eps * np.linalg.norm(Y) * (1 + 1e-12)
    # Claim: ||Y - Y~||^2 = ||Y||^2 - ||C_1||^2 (root holds C_1)
    lhs = err ** 2
    rhs = np.linalg.norm(Y) ** 2 - np.linalg.norm(st.root) ** 2
    assert abs(lhs - rhs) <= 1e-10 * np.linalg.norm(Y) ** 2
    # orthonormal matrix form of every core
    for nd in st.tree.nodes[1:]:
        B = st.basis(nd.id)
        assert np.abs(B.T @ B - np.eye(B.shape[1])).max() < 1e-12


def test_nodewise_errors_sum_bound():
    """Theorem total_approx_error: ||Y - Y~||^2 <= sum of discarded energies, each <= eps_nw^2."""
    rng = np.random.default_rng(7)
    Y = rng.normal(size=(5, 4, 5, 6))
    eps = 0.4
    st = O.bht_l2r(Y, eps)
    thr2 = (eps * np.linalg.norm(Y)) ** 2 / 4
    # leaf on layer 2: discarded energy of its unfolding
    tot = 0.0
    t = st.tree
    for nd in t.layer_nodes(2):
        M = np.moveaxis(Y, nd.mode + 1, 0).reshape(Y.shape[nd.mode + 1], -1)
        P = st.cores[nd.id]
        e = np.linalg.norm(M - P @ (P.T @ M)) ** 2
        assert e <= thr2 * (1 + 1e-12)
        tot += e
    err2 = np.linalg.norm(Y - O.reconstruct(st)) ** 2
    assert err2 <= 4 * thr2 * (1 + 1e-12)


# ---------------------------------------------------------------------------
# HT-RISE: incremental pins (Algorithm 2, Theorems hit_approx_error, hit_past_stream)
# ---------------------------------------------------------------------------

def test_htrise_bound_invariance_orthonormality_c0():
    Y = S.gaussian_bumps(0, 0, 32)
    eps = 1e-3
    st = O.bht_l2r(Y[:8], eps)
    first = O.reconstruct(st, 0, 8).copy()
    for k in range(3):
        Yk = Y[8 + 8 * k:16 + 8 * k]
        info = O.htrise_update(st, Yk, eps)
        Yh = O.reconstruct(st, 8 + 8 * k, 8)
        assert np.linalg.norm(Yk - Yh) <= eps * np.linalg.norm(Yk) * (1 + 1e-12)   # per increment
        # past stream unchanged (Theorem hit_past_stream)
        assert np.abs(O.reconstruct(st, 0, 8) - first).max() <= 1e-13 * np.abs(first).max()
        for nd in st.tree.nodes[1:]:
            B = st.basis(nd.id)
            assert np.abs(B.T @ B - np.eye(B.shape[1])).max() < 1e-12
        if not info.skipped:
            assert all(a >= b for a, b in zip(info.ranks_after[1:], info.ranks_before[1:]))
    Xh = O.reconstruct(st)
    assert np.linalg.norm(Y - Xh) <= eps * np.linalg.norm(Y) * (1 + 1e-12)
    assert st.n_items == 32


def test_skip_projection_norm_identity():
    """Claim orthogonal_reconstructions on the skip path: eps_proj^2 = ||Y - Y~||^2."""
    Y = S.gaussian_bumps(1, 0, 20)
    st = O.bht_l2r(Y[:10], 0.05)
    info = O.htrise_update(st, Y[10:], 0.5)        # loose eps: forced skip
    assert info.skipped
    Yh = O.reconstruct(st, 10, 10)
    assert abs(np.linalg.norm(Y[10:] - Yh) - info.eps_proj) <= 1e-10 * np.linalg.norm(Y[10:])


def test_incremental_equals_one_shot_when_first_batch_spans():
    rng = np.random.default_rng(8)
    Y, _ = tree_d5_exact(rng, (4, 5, 3, 6, 7), RANKS_D5, N=60)
    # eps above sqrt(machine eps): the norm difference of eq. relative_error_threshold
    # cannot resolve errors below ~1.5e-8 ||Y|| in float64
    eps = 1e-6
    st = O.bht_l2r(Y[:40], eps)
    one = O.bht_l2r(Y, eps)
    for a, b in ((40, 50), (50, 60)):
        info = O.htrise_update(st, Y[a:b], eps)
        assert info.skipped
    assert st.ranks()[1:] == one.ranks()[1:]
    assert rel(O.reconstruct(st), O.reconstruct(one)) < 1e-12
    assert rel(O.reconstruct(st), Y) < 1e-12


def test_known_rank_growth():
    """Batch 2 brings directions batch 1 lacks; the updated ranks equal the ranks of the whole stream."""
    rng = np.random.default_rng(9)
    n1, n2, n3 = 6, 7, 5
    A = rand_orth(rng, n1, 4); B = rand_orth(rng, n2, 3); Cm = rand_orth(rng, n3, 3)

    def batch(N, ka, kb):
        core = rng.normal(size=(N, 4, 3, 3))
        core[:, ka:] = 0.0
        core[:, :, kb:] = 0.0
        return np.einsum("nabc,ia,jb,kc->nijk", core, A, B, Cm)

    Y1 = batch(30, 2, 2)          # spans 2 of 4 directions of mode 1, 2 of 3 of mode 2
    Y2 = batch(30, 4, 3)          # spans all
    st = O.bht_l2r(Y1, 1e-10)
    r_before = st.ranks()
    info = O.htrise_update(st, Y2, 1e-10)
    assert not info.skipped
    one = O.bht_l2r(np.concatenate([Y1, Y2]), 1e-10)
    t = st.tree
    leaf = {nd.mode: nd.id for nd in t.nodes if nd.is_leaf}
    assert r_before[leaf[0]] == 2 and r_before[leaf[1]] == 2
    assert st.rank(leaf[0]) == 4 and st.rank(leaf[1]) == 3 and st.rank(leaf[2]) == 3
    assert st.ranks()[1:] == one.ranks()[1:]
    assert rel(O.reconstruct(st), np.concatenate([Y1, Y2])) < 1e-11


# ---------------------------------------------------------------------------
# Band-limit invariants of the spectral stream, compression ratio
# ---------------------------------------------------------------------------

def test_bandlimit_ranks_spectral_field():
    K, n = 3, 12
    Y = S.spectral_field(0, 0, 48, n=n, K=K, dtype=np.float64)
    st = O.bht_l2r(Y, 1e-9)
    t = st.tree
    disc = sum(1 for a in range(-K, K + 1) for b in range(-K, K + 1) if 0 < a * a + b * b <= K * K)
    for nd in t.nodes[1:]:
        if nd.is_leaf:
            assert st.rank(nd.id) == 2 * K + 1          # cos and sin of |kx| = 1..K, plus the mean
    n12 = t.nodes[0].children[0]
    assert st.rank(n12) <= disc + 1                      # functions of (x, y) with kx^2 + ky^2 <= K^2
    assert rel(O.reconstruct(st), Y) < 1e-8


def test_compression_ratio_from_ranks():
    Y = S.gaussian_bumps(2, 0, 12)
    st = O.bht_l2r(Y, 1e-2)
    t = st.tree
    elems = 0
    for nd in t.nodes[1:]:
        if nd.is_leaf:
            elems += t.dims[nd.mode] * st.rank(nd.id)
        else:
            a, b = nd.children
            elems += st.rank(a) * st.rank(b) * st.rank(nd.id)
    c1, c2 = t.nodes[0].children
    elems += st.rank(c1) * st.rank(c2) * 12
    assert O.compression_ratio(st) == 12 * 16 ** 3 / elems


# ---------------------------------------------------------------------------
# App. C: adaptive error budget
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,N,eps", [((6, 7, 5), 4, 0.05), ((4, 5, 3, 6), 5, 0.1), ((3, 4, 5, 3, 4), 6, 0.08),
                                        ((8, 8, 8, 8), 3, 0.03)])
def test_adaptive_budget_keeps_the_bound(dims, N, eps):
    rng = np.random.default_rng(sum(dims) + N)
    Y = rng.normal(size=(N,) + dims)
    Y = Y + 0.5 * np.cumsum(Y, axis=1)
    st = O.bht_l2r(Y, eps, budget="adaptive")
    assert np.linalg.norm(Y - O.reconstruct(st)) <= eps * np.linalg.norm(Y) * (1 + 1e-12)
    for k in range(2):
        Yk = rng.normal(size=(N,) + dims)
        O.htrise_update(st, Yk, eps)
        assert np.linalg.norm(Yk - O.reconstruct(st, st.n_items - N, N)) <= eps * np.linalg.norm(Yk) * (1 + 1e-12)


def test_adaptive_budget_equals_uniform_with_one_layer():
    # d = 2: every truncation is on the first layer, nothing is left to re-budget
    rng = np.random.default_rng(21)
    Y = rng.normal(size=(3, 9, 11))
    a, u = O.bht_l2r(Y, 0.1, budget="adaptive"), O.bht_l2r(Y, 0.1)
    assert a.ranks() == u.ranks()
    np.testing.assert_allclose(O.reconstruct(a), O.reconstruct(u), atol=1e-12)


def test_adaptive_budget_truncates_the_upper_layer_at_least_as_hard():
    # d = 3: layer 2 is identical; layer 1 sees the same intermediate and a tolerance that is the
    # unspent budget spread over its two truncations, never below eps_abs / sqrt(2d - 2)
    rng = np.random.default_rng(22)
    for trial in range(5):
        Y = rng.normal(size=(4, 6, 7, 8)) + np.cumsum(rng.normal(size=(4, 6, 7, 8)), axis=2)
        a, u = O.bht_l2r(Y, 0.2, budget="adaptive"), O.bht_l2r(Y, 0.2)
        ra, ru = a.ranks(), u.ranks()
        t = a.tree
        for nid in t.layers[2]:
            assert ra[nid] == ru[nid]
        for nid in t.layers[1]:
            assert ra[nid] <= ru[nid]


def test_adaptive_budget_tolerance_formula():
    # after layer p: eps_rem^2 = eps_abs^2 - (||Y||^2 - ||C_p||^2), eps_nw = eps_rem / sqrt(svd_rem)
    rng = np.random.default_rng(23)
    C = rng.normal(size=(5, 6))
    norm2 = float(np.sum(C * C)) + 2.0                      # 2.0 of energy already removed
    got = OB._adaptive_eps_nw(9.0, norm2, C, 4)
    assert abs(got - np.sqrt((9.0 - 2.0) / 4)) < 1e-12
    assert OB._adaptive_eps_nw(1.0, norm2, C, 4) == 0.0      # budget already spent: nothing more may be cut


def test_remaining_truncation_counts_of_a_five_mode_tree():
    # Fig. 2 style tree of 5 modes: layer 1 {1,2,3},{4,5}; layer 2 {1,2},{3},{4},{5}; layer 3 {1},{2}
    t = O.dimension_tree((3, 4, 5, 6, 7))
    assert [len(l) for l in t.layers] == [1, 2, 4, 2]
    assert OB._svds_above(t, 4) == 8       # before layer 3: all 2d - 2 truncations remain
    assert OB._svds_above(t, 3) == 6       # after layer 3: layers 2 and 1
    assert OB._svds_above(t, 2) == 2       # after layer 2: layer 1


# ---------------------------------------------------------------------------
# Decoding of latent items and the relative test error (eq. htucker_reconstruction with the
# orthonormal frames of Sec. 3; Step 1 of Algorithm 2 as the encoder)
# ---------------------------------------------------------------------------

def _small_state(seed, dims=(2, 3, 2, 3), eps=0.3, N=6):
    rng = np.random.default_rng(seed)
    Y = rng.normal(size=(N,) + dims) + np.cumsum(rng.normal(size=(N,) + dims), axis=1)
    return O.bht_l2r(Y, eps), Y


def test_decode_of_a_unit_latent_by_explicit_loops():
    # tree of (2,3,2,3): layer 1 {1,2},{3,4}; layer 2 the leaves. decode(e_ij) is the outer product of the
    # two layer-1 frames' columns i and j, each frame (U_a (x) U_b) B written out index by index
    st, _ = _small_state(31)
    t = st.tree
    l1 = t.layers[1]
    cores = st.cores
    frames = []
    for nid in l1:
        a, b = t.nodes[nid].children
        Ua, Ub, Bt = cores[a], cores[b], cores[nid]
        na, nb = Ua.shape[0], Ub.shape[0]
        F = np.zeros((na, nb, Bt.shape[2]))
        for x in range(na):
            for y in range(nb):
                for k in range(Bt.shape[2]):
                    F[x, y, k] = sum(Ua[x, p] * Ub[y, q] * Bt[p, q, k]
                                     for p in range(Ua.shape[1]) for q in range(Ub.shape[1]))
        frames.append(F)
    r11, r12 = frames[0].shape[2], frames[1].shape[2]
    for i in range(r11):
        for j in range(r12):
            Z = np.zeros((1, r11, r12))
            Z[0, i, j] = 1.0
            want = np.einsum("ab,cd->abcd", frames[0][:, :, i], frames[1][:, :, j])
            assert np.abs(O.decode(st, Z)[0] - want).max() < 1e-13


def test_decode_is_an_isometry_and_the_adjoint_of_projection():
    st, _ = _small_state(32, dims=(3, 4, 5, 2, 3), eps=0.2, N=9)
    rng = np.random.default_rng(33)
    r = st.ranks()
    Z = rng.normal(size=(7, r[1], r[2]))
    X = rng.normal(size=(7,) + st.tree.dims)
    D = O.decode(st, Z)
    for n in range(7):      # orthonormal frames: every item keeps its norm
        assert abs(np.linalg.norm(D[n]) - np.linalg.norm(Z[n])) < 1e-12 * np.linalg.norm(Z[n])
    assert abs(np.sum(D * X) - np.sum(Z * O.project(st, X))) < 1e-11 * np.linalg.norm(Z) * np.linalg.norm(X)


def test_relative_test_error_closed_forms():
    # items that are sums of three separable terms plus 5 % noise: the frames keep a small subspace
    rng = np.random.default_rng(34)
    dims = (4, 5, 4, 5)
    Y = sum(np.einsum("n,a,b,c,d->nabcd", *[rng.normal(size=m) for m in (12,) + dims]) for _ in range(3))
    Y = Y + 0.05 * np.linalg.norm(Y) / np.sqrt(Y.size) * rng.normal(size=Y.shape)
    st = O.bht_l2r(Y, 0.25)
    r = st.ranks()
    k, n = r[1] * r[2], int(np.prod(st.tree.dims))
    assert k < n // 4
    # items drawn from the represented subspace are represented exactly
    assert O.relative_test_error(st, O.decode(st, rng.normal(size=(5, r[1], r[2])))) < 1e-13
    # isotropic Gaussian items keep k/n of their energy on average: RTE^2 -> 1 - k/n (chi-square with
    # k of N n degrees of freedom; 4000 items put the relative spread of the estimate near 1e-3)
    rte = O.relative_test_error(st, rng.normal(size=(4000,) + st.tree.dims))
    assert abs(rte ** 2 - (1 - k / n)) < 0.02 * (1 - k / n)
    # the accumulated batch itself: BHT-l2r's root is the projection of the batch, so each item's error is
    # that of its stored approximation; the average of eq. generalization_performance, item by item
    rec = O.reconstruct(st)
    want = np.mean([np.linalg.norm(rec[i] - Y[i]) / np.linalg.norm(Y[i]) for i in range(Y.shape[0])])
    got, errs = O.relative_test_error(st, Y, per_item=True)
    assert abs(got - want) < 1e-12
    # the aggregate error meets the bound of Corollary bht_leaves_to_root; individual items may not
    assert np.sqrt(np.sum((errs * np.linalg.norm(Y.reshape(12, -1), axis=1)) ** 2)) <= 0.25 * np.linalg.norm(Y) * (1 + 1e-12)
    # an all-zero item counts 0 and leaves the others' average unchanged
    Z = np.concatenate([Y[:3], np.zeros_like(Y[:1])])
    assert abs(O.relative_test_error(st, Z) - np.mean(errs[:3]) * 3 / 4) < 1e-12


def test_reduction_ratio_and_normalisations():
    st, _ = _small_state(36, dims=(4, 5, 6), eps=0.2, N=5)
    r = st.ranks()
    assert O.reduction_ratio(st) == 120 / (r[1] * r[2])
    rng = np.random.default_rng(37)
    Y = rng.normal(size=(6, 2, 5, 7)) * rng.uniform(0.1, 10, size=(6, 2, 1, 1)) + 3.0
    for kind in ("maxabs", "unitvec", "zscore", "none"):
        Yn, P = O.normalize(Y, kind, groups=12)                 # per item and physical quantity
        G = Yn.reshape(12, -1)
        if kind == "maxabs":
            assert np.allclose(np.abs(G).max(axis=1), 1.0, atol=1e-15)
        elif kind == "unitvec":
            assert np.allclose(np.linalg.norm(G, axis=1), 1.0, atol=1e-14)
        elif kind == "zscore":
            assert np.allclose(G.mean(axis=1), 0.0, atol=1e-14) and np.allclose(G.std(axis=1), 1.0, atol=1e-14)
        else:
            assert np.array_equal(Yn, Y)
        assert np.allclose((G * P[:, 1:2] + P[:, 0:1]).reshape(Y.shape), Y, rtol=0, atol=1e-13)
    Yc = np.ones((2, 3, 4))
    Yn, P = O.normalize(Yc, "zscore")                            # constant item: scale falls back to 1
    assert np.array_equal(P[:, 1], [1.0, 1.0]) and np.array_equal(Yn, np.zeros_like(Yc))


# ---------------------------------------------------------------------------
# Plain HT baseline: the batch as the last leaf (Fig. htucker_as_node), leaves-to-root of Sec. 2.3.1
# ---------------------------------------------------------------------------

def test_plain_ht_two_mode_items_are_the_truncated_svd_of_the_matricisation():
    # items of 3 x 4: tree over (3, 4, N) = {1,2},{N}; {1},{2}. Items drawn from a 5-dimensional space
    # plus 1e-4 noise keep both leaves at full rank, so the layer-1 SVD acts on (n_1 n_2) x N through an
    # orthogonal change of basis: the result is the Eckart-Young truncation of that matrix (LAPACK)
    rng = np.random.default_rng(41)
    N = 50
    A = rng.normal(size=(12, 5)) @ rng.normal(size=(5, N))
    A = A + 1e-4 * rng.normal(size=A.shape)
    Y = A.T.reshape(N, 3, 4)
    st = O.ht_l2r(Y, 1e-2)
    r = st.ranks()
    t = st.tree
    assert [r[nid] for nid in t.layers[2]] == [3, 4]
    assert r[t.layers[1][0]] == r[t.layers[1][1]] == 5
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    best = (U[:, :5] * s[:5]) @ Vt[:5]
    assert rel(O.ht_items(st).reshape(N, 12).T, best) < 1e-12
    assert np.allclose(np.diag(st.root[:, :, 0]), s[:5], rtol=1e-12, atol=0)


def test_plain_ht_recovers_known_ranks():
    # a tensor built index by index from a chosen HT over (4, 5, 6, N=7): {1,2},{3,N}; leaf ranks 2,3,2,3
    rng = np.random.default_rng(42)
    U1, U2, U3, U4 = rand_orth(rng, 4, 2), rand_orth(rng, 5, 3), rand_orth(rng, 6, 2), rand_orth(rng, 7, 3)
    B12 = rand_orth(rng, 6, 2).reshape(2, 3, 2)
    B34 = rand_orth(rng, 6, 2).reshape(2, 3, 2)
    S0 = np.diag([3.0, 0.5])
    T = np.einsum("ai,bj,ijk,kl,cm,dn,mnl->abcd", U1, U2, B12, S0, U3, U4, B34)
    Y = np.moveaxis(T, -1, 0)
    st = O.ht_l2r(Y, 1e-10)
    t = st.tree
    r = st.ranks()
    assert [r[nid] for nid in t.layers[1]] == [2, 2]
    assert [r[t.leaf_of_mode[m]] for m in range(4)] == [2, 3, 2, 3]
    assert rel(O.ht_items(st), Y) < 1e-12
    assert np.allclose(np.diag(st.root[:, :, 0]), [3.0, 0.5], rtol=1e-12)


@pytest.mark.parametrize("eps", [0.3, 0.1, 0.03])
def test_plain_ht_error_bound_and_tolerance(monkeypatch, eps):
    rng = np.random.default_rng(43)
    Y = np.cumsum(np.cumsum(rng.normal(size=(9, 5, 6, 7, 4)), axis=2), axis=3)
    seen = []
    real = OB.truncated_left_svd
    monkeypatch.setattr(OB, "truncated_left_svd", lambda M, e, rmin=1: (seen.append(e), real(M, e, rmin))[1])
    st = O.ht_l2r(Y, eps)
    # d = 4 item modes plus the batch: 2 (d + 1) - 3 = 7 truncations share the budget
    assert all(abs(e - eps * np.linalg.norm(Y) / np.sqrt(7)) < 1e-12 * np.linalg.norm(Y) for e in seen)
    assert len(seen) == 2 * 5 - 2 - 2          # every non-root node but the two of the last SVD
    assert np.linalg.norm(Y - O.ht_items(st)) <= eps * np.linalg.norm(Y) * (1 + 1e-12)
    # nested orthonormal frames (orthonormal leaves and reshaped transfer cores)
    for nd in st.tree.non_root():
        Bm = st.basis(nd.id)
        assert np.abs(Bm.T @ Bm - np.eye(Bm.shape[1])).max() < 1e-12

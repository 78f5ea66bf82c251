"""GPU path against the FP64 oracle, element by element, through the C ABI.

Parity definition (FP64 GPU path):
  * ranks equal to the oracle's, unless the oracle's discarded energy at that
    node is within TIE_REL * ||Y||^2 of eps_nw^2 (then either rank is right);
  * ||Y~_gpu - Y~_oracle|| / ||Y|| <= RECON_TOL when the ranks agree;
  * ||Y - Y~_gpu|| <= eps ||Y|| (Corollary bht_leaves_to_root, Problem 2),
    with a relative slack of 1e-9 for FP64 rounding;
  * the skip decision of HT-RISE equals the oracle's away from the threshold;
  * past items reconstruct identically after later updates (Theorem hit_past_stream).
"""
import numpy as np
import pytest

import bht_synth as S
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RECON_TOL = 1e-10
TIE_REL = 1e-10


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


def recon(B, st, first, count):
    out = B.ht_reconstruct(st, first, count, dtype="float64")
    torch.cuda.synchronize()
    return out.cpu().numpy()


def ranks_match(gpu_ranks, ost):
    return gpu_ranks[1:] == ost.ranks()[1:]


def run_stream(B, batches, eps, precision="fp64", host=False):
    """Run BHT-l2r on the first batch, HT-RISE on the rest, on GPU and in the oracle."""
    tree = B.bht_tree_create_balanced(batches[0].shape[1:])
    src = (lambda y: y) if host else to_dev
    st = B.bht_l2r(tree, src(batches[0]), eps, precision=precision)
    ost = O.bht_l2r(batches[0], eps)
    infos = []
    for Yk in batches[1:]:
        gi = B.htrise_update(st, src(Yk), eps, precision=precision)
        oi = O.htrise_update(ost, Yk, eps)
        infos.append((gi, oi))
    B.bht_tree_destroy(tree)
    return st, ost, infos


# ---------------------------------------------------------------------------
# small shapes: several tiles, ragged tails, N = 1, d = 2 .. 5
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dims,N,eps", [
    ((7, 9), 1, 0.05),
    ((70, 33), 5, 0.01),
    ((5, 6, 7), 3, 0.1),
    ((16, 16, 16), 8, 1e-3),
    ((13, 67, 11), 4, 1e-2),
    ((4, 5, 3, 6), 6, 0.05),
    ((3, 4, 5, 3, 4), 9, 0.02),
])
def test_bht_l2r_matches_oracle(B, dims, N, eps):
    rng = np.random.default_rng(sum(dims) * 31 + N)
    Y = rng.normal(size=(N,) + dims)
    Y = Y + 0.5 * np.cumsum(Y, axis=1) if len(dims) > 1 else Y
    tree = B.bht_tree_create_balanced(dims)
    st = B.bht_l2r(tree, to_dev(Y), eps)
    ost = O.bht_l2r(Y, eps)
    g = B.bht_get_ranks(st)
    assert g[0] == N
    Yg = recon(B, st, 0, N)
    assert np.linalg.norm(Y - Yg) <= eps * np.linalg.norm(Y) * (1 + 1e-9)
    assert ranks_match(g, ost), (g, ost.ranks())
    assert rel(Yg, O.reconstruct(ost)) <= RECON_TOL * max(1.0, np.linalg.norm(Y) / np.linalg.norm(O.reconstruct(ost)))
    # root norm identity of the orthogonal reconstruction claim
    root = B.bht_get_root(st, 0, N)
    assert abs(np.linalg.norm(root) ** 2 - np.linalg.norm(Yg) ** 2) <= 1e-10 * np.linalg.norm(Y) ** 2
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_fp32_input_and_host_pointer(B):
    Y = S.gaussian_bumps(3, 0, 6).astype(np.float32)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st_dev = B.bht_l2r(tree, to_dev(Y), 1e-2)
    st_host = B.bht_l2r(tree, Y, 1e-2)           # host numpy pointer: staged by the library
    assert B.bht_get_ranks(st_dev) == B.bht_get_ranks(st_host)
    a, b = recon(B, st_dev, 0, 6), recon(B, st_host, 0, 6)
    # FP64 atomics make the Gram summation order vary from run to run: equal up to rounding
    assert rel(a, b) < 1e-12
    ost = O.bht_l2r(Y.astype(np.float64), 1e-2)
    assert ranks_match(B.bht_get_ranks(st_dev), ost)
    assert rel(a, O.reconstruct(ost)) <= RECON_TOL
    out_host = np.empty_like(Y)
    B.ht_reconstruct(st_host, 0, 6, out=out_host)
    assert rel(out_host, a) < 1e-6
    B.bht_state_destroy(st_dev)
    B.bht_state_destroy(st_host)
    B.bht_tree_destroy(tree)


# ---------------------------------------------------------------------------
# the 16^3 Gaussian-bump stream in full: BHT-l2r on 8 items, 3 HT-RISE updates of 8
# ---------------------------------------------------------------------------

def test_gaussian_bump_stream_matches_oracle(B):
    Y = S.gaussian_bumps(0, 0, 32)
    eps = 1e-3
    batches = [Y[:8], Y[8:16], Y[16:24], Y[24:32]]
    st, ost, infos = run_stream(B, batches, eps)
    for gi, oi in infos:
        assert gi.skipped == oi.skipped
        assert abs(gi.eps_proj - oi.eps_proj) <= 1e-7 * gi.norm_y
    assert ranks_match(B.bht_get_ranks(st), ost)
    Yg = recon(B, st, 0, 32)
    assert rel(Yg, O.reconstruct(ost)) <= RECON_TOL * 10
    for k in range(4):
        Yk, Gk = Y[8 * k:8 * k + 8], Yg[8 * k:8 * k + 8]
        assert np.linalg.norm(Yk - Gk) <= eps * np.linalg.norm(Yk) * (1 + 1e-9)
    # latent encoding of unseen items equals the oracle's projection
    Yt = S.gaussian_bumps(0, 100, 4)
    enc = B.ht_encode(st, to_dev(Yt))
    dec = B.ht_decode(st, enc, dtype="float64").cpu().numpy()
    # the cores agree up to rotations, which encode-then-decode cancels: compare element by element
    dec_o = O.decode(ost, O.project(ost, Yt))
    assert np.abs(dec - dec_o).max() <= RECON_TOL * 10 * np.abs(Yt).max()
    B.bht_state_destroy(st)


def test_past_stream_invariance_on_gpu(B):
    Y = S.gaussian_bumps(5, 0, 24)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, to_dev(Y[:6]), 1e-3)
    first = recon(B, st, 0, 6)
    for k in range(3):
        B.htrise_update(st, to_dev(Y[6 + 6 * k:12 + 6 * k]), 1e-3)
        again = recon(B, st, 0, 6)
        assert np.abs(again - first).max() <= 1e-12 * np.abs(first).max()
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_known_rank_growth_on_gpu(B):
    rng = np.random.default_rng(9)

    def orth(r, c):
        return np.linalg.qr(rng.normal(size=(r, c)))[0]

    A, Bm, Cm = orth(6, 4), orth(7, 3), orth(5, 3)

    def batch(N, ka, kb):
        core = rng.normal(size=(N, 4, 3, 3))
        core[:, ka:] = 0.0
        core[:, :, kb:] = 0.0
        return np.einsum("nabc,ia,jb,kc->nijk", core, A, Bm, Cm)

    Y1, Y2 = batch(30, 2, 2), batch(30, 4, 3)
    st, ost, infos = run_stream(B, [Y1, Y2], 1e-6)
    assert not infos[0][0].skipped
    g = B.bht_get_ranks(st)
    assert ranks_match(g, ost)
    t = O.dimension_tree(Y1.shape[1:])
    leaf = {nd.mode: nd.id for nd in t.nodes if nd.is_leaf}
    assert (g[leaf[0]], g[leaf[1]], g[leaf[2]]) == (4, 3, 3)
    Yg = recon(B, st, 0, 60)
    assert rel(Yg, np.concatenate([Y1, Y2])) < 1e-9
    B.bht_state_destroy(st)


def test_non_finite_input_is_rejected(B):
    Y = S.gaussian_bumps(1, 0, 4)
    Y[2, 3, 4, 5] = np.nan
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    with pytest.raises(B.BHTError) as e:
        B.bht_l2r(tree, to_dev(Y), 1e-2)
    assert e.value.status == 5
    B.bht_tree_destroy(tree)

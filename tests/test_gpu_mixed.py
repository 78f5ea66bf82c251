"""Mixed-precision GPU path (tcgen05 split-TF32 mode products, FP32 SIMT
contractions, FP32 Grams summed in FP64, FP64 eigensolves) against the FP64
oracle, through the C ABI.

Tolerances follow from the arithmetic: the split-TF32 products carry a
relative error of about 2^-20, the FP32 Grams about 1e-7 relative per entry.
  * a node rank may differ from the oracle's only where the oracle's
    discarded energy lies within TIE * ||Y||^2 of eps_nw^2 (TIE = 1e-6);
  * with equal ranks, ||Y~_gpu - Y~_oracle|| <= RECON * ||Y|| (RECON = 1e-4);
  * ||Y - Y~_gpu|| <= eps ||Y|| (1 + 1e-4) for every batch.
"""
import numpy as np
import pytest

import bht_synth as S
import oracle as O
import oracle.bht_oracle as OB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIE = 1e-6
RECON = 1e-4


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


class Recorder:
    """Records every truncation the oracle makes: (squared singular values, eps_nw^2, chosen rank)."""

    def __init__(self, monkeypatch):
        self.calls = []
        orig = OB.truncated_left_svd

        def rec(M, eps_nw, rmin=1):
            U, s2 = orig(M, eps_nw, rmin)
            self.calls.append((s2, eps_nw * eps_nw, U.shape[1]))
            return U, s2

        monkeypatch.setattr(OB, "truncated_left_svd", rec)

    def near_tie(self, norm2):
        """True when some truncation's discarded energy is within TIE*||Y||^2 of its threshold."""
        for s2, thr, r in self.calls:
            tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])
            for q in (r - 1, r):
                if 0 <= q < len(tail) and abs(tail[q] - thr) <= TIE * norm2:
                    return True
        return False


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / np.linalg.norm(b))


def to_dev(Y):
    return torch.from_numpy(np.ascontiguousarray(Y)).cuda()


def recon(B, st, first, count):
    return B.ht_reconstruct(st, first, count, dtype="float64").cpu().numpy()


@pytest.mark.parametrize("dims,N,eps", [
    ((16, 16, 16), 8, 1e-2),
    ((13, 68, 12), 4, 1e-2),
    ((4, 5, 3, 6), 6, 0.05),
    ((8, 12, 16, 4, 8), 5, 0.02),
    ((64, 64), 3, 1e-2),
])
def test_mixed_bht_l2r_matches_oracle(B, monkeypatch, dims, N, eps):
    rng = np.random.default_rng(sum(dims) + 7 * N)
    Y = rng.normal(size=(N,) + dims)
    Y = (Y + 0.5 * np.cumsum(Y, axis=1)).astype(np.float32)
    rec = Recorder(monkeypatch)
    ost = O.bht_l2r(Y.astype(np.float64), eps)
    tree = B.bht_tree_create_balanced(dims)
    st = B.bht_l2r(tree, to_dev(Y), eps, precision="mixed")
    g = B.bht_get_ranks(st)
    Yg = recon(B, st, 0, N)
    n2 = float(np.sum(Y.astype(np.float64) ** 2))
    assert np.linalg.norm(Y - Yg) <= eps * np.sqrt(n2) * (1 + 1e-4)
    if g[1:] != ost.ranks()[1:]:
        assert rec.near_tie(n2), (g, ost.ranks())
    else:
        assert rel(Yg, O.reconstruct(ost)) <= RECON
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


def test_mixed_gaussian_bump_stream(B, monkeypatch):
    Y = S.gaussian_bumps(0, 0, 32).astype(np.float32)
    Y64 = Y.astype(np.float64)
    eps = 1e-2
    rec = Recorder(monkeypatch)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, to_dev(Y[:8]), eps, precision="mixed")
    ost = O.bht_l2r(Y64[:8], eps)
    for k in range(1, 4):
        gi = B.htrise_update(st, to_dev(Y[8 * k:8 * k + 8]), eps, precision="mixed")
        oi = O.htrise_update(ost, Y64[8 * k:8 * k + 8], eps)
        # the skip decision agrees unless the projection error sits at the threshold
        if abs(oi.eps_proj - oi.eps_des) > 1e-4 * gi.norm_y:
            assert gi.skipped == oi.skipped
    Yg = recon(B, st, 0, 32)
    for k in range(4):
        assert np.linalg.norm(Y64[8 * k:8 * k + 8] - Yg[8 * k:8 * k + 8]) <= \
            eps * np.linalg.norm(Y64[8 * k:8 * k + 8]) * (1 + 1e-4)
    if B.bht_get_ranks(st)[1:] == ost.ranks()[1:]:
        assert rel(Yg, O.reconstruct(ost)) <= RECON
    else:
        assert rec.near_tie(float(np.sum(Y64 ** 2)))
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spectral_field_full_size_increments(B, monkeypatch, precision):
    """The 64^3 advected spectral field at its full size: BHT-l2r on 32 snapshots, two HT-RISE updates of 32."""
    eps = 1e-2
    Y = S.spectral_field(0, 0, 96)
    Y64 = Y.astype(np.float64)
    rec = Recorder(monkeypatch)
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, to_dev(Y[:32]), eps, precision=precision)
    ost = O.bht_l2r(Y64[:32], eps)
    infos = []
    for k in (1, 2):
        gi = B.htrise_update(st, to_dev(Y[32 * k:32 * k + 32]), eps, precision=precision)
        oi = O.htrise_update(ost, Y64[32 * k:32 * k + 32], eps)
        infos.append((gi, oi))
        if abs(oi.eps_proj - oi.eps_des) > 1e-4 * gi.norm_y:
            assert gi.skipped == oi.skipped
        assert abs(gi.eps_proj - oi.eps_proj) <= 1e-3 * gi.norm_y
    Yg = B.ht_reconstruct(st, 0, 96, dtype="float32")
    Yd = to_dev(Y)
    for k in range(3):
        err = float(torch.linalg.vector_norm((Yg[32 * k:32 * k + 32] - Yd[32 * k:32 * k + 32]).double()))
        assert err <= eps * float(torch.linalg.vector_norm(Yd[32 * k:32 * k + 32].double())) * (1 + 1e-4)
    g = B.bht_get_ranks(st)
    if g[1:] == ost.ranks()[1:]:
        # sampled items compared with the oracle's reconstruction
        tol = 1e-9 if precision == "fp64" else RECON
        for item in (0, 45, 95):
            a = B.ht_reconstruct(st, item, 1, dtype="float64").cpu().numpy()[0]
            b = O.reconstruct(ost, item, 1)[0]
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(Y64[item])
    else:
        assert rec.near_tie(float(np.sum(Y64[:32] ** 2)))
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)

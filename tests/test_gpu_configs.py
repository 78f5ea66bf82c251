"""Streams shaped like the paper's workloads, GPU path against the FP64 oracle through the C ABI.

* multi-variable simulation stream: 5 variables x 48^3, increments of uneven sizes drawn from 1..64,
  eps = 1e-3 (a 4-mode tree {1,2},{3,4});
* the 64^3 advected spectral field at the tight tolerance eps = 1e-4;
* a two-way stream whose spectrum is graded over twelve decades, at eps = 1e-6;
* the 24^5 Chebyshev sensor stream: a few items against the oracle, one full increment of 64 items
  (2.04 GB) against the oracle item by item, and two full increments checked through properties
  that hold at any size: the error bound per
  increment, orthonormal cores, leaf ranks bounded by the polynomial degree, and the decode of
  sampled items against a host contraction of the same cores.

Tolerances: mixed path ranks equal unless the oracle's discarded energy lies within TIE * ||Y||^2
of its threshold, reconstructions within 1e-4 * ||Y||; both ||Y - Y~|| <= eps ||Y|| (1 + 1e-4).
FP64 path: ranks equal, reconstructions within 1e-9 + 10 sum_t theta_t sigma_r / ||M_t|| over the
truncations t, theta_t = min(1, n_t eps_mach sigma_1^2 / (sigma_r^2 - sigma_{r+1}^2)). The GPU takes
eigenvectors of an n_t x n_t Gram matrix, whose kept subspace is fixed to about n_t eps_mach ||G||
over the eigenvalue gap at the cut (theta_t), and a rotation by theta_t between the last kept and the
first discarded direction moves sigma_r theta_t of the data; the oracle's SVD is far more accurate
there. With well-separated cuts the bound is below 1e-9; at eps = 1e-4 the band-limited field cuts
node {1,2} between eigenvalues 3 % apart at 1e-9 of the largest, where it is not.
"""
import numpy as np
import pytest

import bht_synth as S
import oracle as O
import oracle.bht_oracle as OB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIE = {"fp64": 1e-10, "mixed": 1e-6}
RECON = {"fp64": 1e-9, "mixed": 1e-4}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


class Recorder:
    """Every truncation the oracle makes: (squared singular values, threshold, chosen rank)."""

    def __init__(self, monkeypatch):
        self.calls = []
        orig = OB.truncated_left_svd

        def rec(M, eps_nw, rmin=1):
            U, s2 = orig(M, eps_nw, rmin)
            self.calls.append((s2, eps_nw * eps_nw, U.shape[1]))
            return U, s2

        monkeypatch.setattr(OB, "truncated_left_svd", rec)

    def gram_bound(self):
        """sum over truncations of theta_t * sigma_r / ||M_t|| (module docstring)."""
        tot = 0.0
        for s2, thr, r in self.calls:
            if 0 < r < len(s2) and s2[0] > 0:
                theta = min(1.0, len(s2) * np.finfo(np.float64).eps * s2[0] / max(s2[r - 1] - s2[r], 1e-300))
                tot += theta * np.sqrt(s2[r - 1] / np.sum(s2))
        return tot

    def near_tie(self, norm2, tie):
        for s2, thr, r in self.calls:
            tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])
            for q in (r - 1, r):
                if 0 <= q < len(tail) and abs(tail[q] - thr) <= tie * norm2:
                    return True
        return False


def to_dev(Y):
    return torch.from_numpy(np.ascontiguousarray(Y)).cuda()


def check_stream(B, monkeypatch, batches, eps, precision, sample_items, budget="uniform"):
    """BHT-l2r on the first batch, HT-RISE on the rest, GPU and oracle side by side."""
    rec = Recorder(monkeypatch)
    tree = B.bht_tree_create_balanced(batches[0].shape[1:])
    st = B.bht_l2r(tree, to_dev(batches[0]), eps, precision=precision, budget=budget)
    ost = O.bht_l2r(batches[0].astype(np.float64), eps, budget=budget)
    for Yk in batches[1:]:
        gi = B.htrise_update(st, to_dev(Yk), eps, precision=precision)
        oi = O.htrise_update(ost, Yk.astype(np.float64), eps)
        if abs(oi.eps_proj - oi.eps_des) > 1e-4 * gi.norm_y:
            assert gi.skipped == oi.skipped
        assert abs(gi.eps_proj - oi.eps_proj) <= 1e-3 * gi.norm_y
    first = 0
    for Yk in batches:
        Yg = B.ht_reconstruct(st, first, len(Yk), dtype="float64")
        Yd = to_dev(Yk.astype(np.float64))
        err = float(torch.linalg.vector_norm(Yg - Yd))
        assert err <= eps * float(torch.linalg.vector_norm(Yd)) * (1 + 1e-4)
        first += len(Yk)
    norm2 = sum(float(np.sum(Yk.astype(np.float64) ** 2)) for Yk in batches)
    if B.bht_get_ranks(st)[1:] == ost.ranks()[1:]:
        allY = np.concatenate(batches).astype(np.float64)
        tol = RECON[precision] + (10.0 * rec.gram_bound() if precision == "fp64" else 0.0)
        for item in sample_items:
            a = B.ht_reconstruct(st, item, 1, dtype="float64").cpu().numpy()[0]
            b = O.reconstruct(ost, item, 1)[0]
            assert np.linalg.norm(a - b) <= tol * np.linalg.norm(allY[item])
    else:
        assert rec.near_tie(norm2, TIE[precision]), (B.bht_get_ranks(st), ost.ranks())
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multivariable_stream_uneven_increments(B, monkeypatch, precision):
    sizes = [int(x) for x in S.increment_sizes(0, 4)]          # uneven sizes from 1..64
    Y = S.multivar_field(0, 0, sum(sizes))                     # [N, 5, 48, 48, 48]
    batches = np.split(Y, np.cumsum(sizes)[:-1])
    check_stream(B, monkeypatch, batches, 1e-3, precision, sample_items=(0, sizes[0], sum(sizes) - 1))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_spectral_field_tight_tolerance(B, monkeypatch, precision):
    Y = S.spectral_field(0, 0, 64)
    check_stream(B, monkeypatch, [Y[:32], Y[32:]], 1e-4, precision, sample_items=(0, 40, 63))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chebyshev_sensor_small(B, monkeypatch, precision):
    Y = S.chebyshev_sensor(0, 0, 6)
    check_stream(B, monkeypatch, [Y[:3], Y[3:]], 1e-2, precision, sample_items=(0, 5))


def test_graded_spectrum_tight_tolerance(B, monkeypatch):
    """A mode-1 spectrum graded over twelve decades at eps = 1e-6: BHT-l2r keeps 284 of 400 directions,
    68 of them with eigenvalues below 1e-9 of the largest and gaps near 1e-13 of it (one chain for the
    cluster Gram-Schmidt); the first update expands the leaf by a residual of the same grading, and the
    last batch lies in the span already kept (a skip). The tail sums at the cuts sit at least 12 % away
    from their thresholds, so the ranks are well defined in FP64."""
    batches = S.graded_stream(0)
    check_stream(B, monkeypatch, batches, 1e-6, "fp64", sample_items=(0, 47, 60, 143))


def _host_decode(B, st, dims, item):
    """One item decoded on the host in FP64 from the cores the library holds (eq. htucker_reconstruction)."""
    tree = OB.dimension_tree(dims)
    ranks = B.bht_get_ranks(st)
    root = B.bht_get_root(st, item, 1)[0]                     # [r11, r12]

    def expand(nid):                                           # basis of node nid: [prod of its modes' dims, r]
        nd = tree.nodes[nid]
        core = B.bht_get_core(st, nid)
        if nd.is_leaf:
            return core.reshape(dims[nd.mode], ranks[nid])
        a, b = nd.children
        Ua, Ub = expand(a), expand(b)
        G = core.reshape(ranks[a], ranks[b], ranks[nid])
        return np.einsum("ia,jb,abr->ijr", Ua, Ub, G).reshape(Ua.shape[0] * Ub.shape[0], ranks[nid])

    a, b = tree.nodes[0].children
    return (expand(a) @ root @ expand(b).T).reshape(dims)


def test_chebyshev_sensor_full_increment_matches_oracle(B, monkeypatch):
    """One whole increment of the 24^5 sensor stream (64 items, 2.04 GB of fp32; 4.1 GB in the FP64 oracle),
    mixed path against the oracle item by item: every one of the 64 items is decoded on both sides."""
    Y = S.chebyshev_sensor(0, 0, 64)
    check_stream(B, monkeypatch, [Y], 1e-2, "mixed", sample_items=range(64))


def test_chebyshev_sensor_full_increments_properties(B):
    """Two increments of 64 items of 24^5 (the stream's increment size), mixed path."""
    eps = 1e-2
    dims = (24,) * 5
    tree = B.bht_tree_create_balanced(dims)
    st = None
    Ys = []
    for k in range(2):
        Yk = to_dev(S.chebyshev_sensor(0, 64 * k, 64))
        Ys.append(Yk)
        if k == 0:
            st = B.bht_l2r(tree, Yk, eps, precision="mixed")
        else:
            B.htrise_update(st, Yk, eps, precision="mixed")
    for k, Yk in enumerate(Ys):
        Yg = B.ht_reconstruct(st, 64 * k, 64, dtype="float32")
        err = float(torch.linalg.vector_norm((Yg - Yk).double()))
        assert err <= eps * float(torch.linalg.vector_norm(Yk.double())) * (1 + 1e-4)
        del Yg
    otree = OB.dimension_tree(dims)
    ranks = B.bht_get_ranks(st)
    for nd in otree.nodes[1:]:
        U = B.bht_get_core(st, nd.id).reshape(-1, ranks[nd.id])
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-10
        if nd.is_leaf:
            assert ranks[nd.id] <= 7                            # degree <= 6 Chebyshev series per mode
    for item in (0, 70, 127):
        # the mixed decode runs its mode products in split TF32 / FP32: about 2^-20 relative per level
        a = B.ht_reconstruct(st, item, 1, dtype="float64").cpu().numpy()[0]
        b = _host_decode(B, st, dims, item)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["spectral", "multivar", "random5"])
def test_adaptive_error_budget(B, monkeypatch, precision, case):
    """App. C: the unspent budget moves up the tree; GPU and oracle take the same truncations."""
    if case == "spectral":
        Y = S.spectral_field(3, 0, 48, n=32)
        batches = [Y[:16], Y[16:32], Y[32:]]
        eps = 2e-2
    elif case == "multivar":
        Y = S.multivar_field(1, 0, 20, n=16)
        batches = [Y[:8], Y[8:13], Y[13:]]
        eps = 1e-2
    else:
        rng = np.random.default_rng(5)
        Y = rng.normal(size=(18, 4, 5, 6, 3, 4))
        Y = (Y + 0.7 * np.cumsum(Y, axis=2)).astype(np.float32)
        batches = [Y[:6], Y[6:12], Y[12:]]
        eps = 0.1
    check_stream(B, monkeypatch, batches, eps, precision, sample_items=(0, len(Y) - 1), budget="adaptive")

"""The bounded device-side waits give up cleanly, through the C ABI.

A host-side test hook (bht_debug_withhold_barrier) makes CTA 0 of the next multi-CTA tridiagonalisation
withhold its first grid-barrier arrival and shortens the wait limit to 20 ms. No GPU fault is involved:
every waiting CTA gives up, writes BHT_ETIMEOUT into the call's status word and returns; the call fails
with that code, the context stays usable, and htrise_update leaves its state exactly as it was (the new
cores live in a shadow copy until the commit).
"""
import numpy as np
import pytest

import bht_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BHT_ETIMEOUT = 6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    yield B
    B.bht_debug_withhold_barrier(0, 1)


def _gram(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n + 3)) * np.logspace(0, -3, n)[:, None]
    return X @ X.T


def test_eigensolver_wait_gives_up_and_the_context_recovers(B):
    G = _gram(300, 1)
    B.bht_debug_withhold_barrier(1, 20)
    with pytest.raises(B.BHTError) as e:
        B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), 5)
    assert e.value.status == BHT_ETIMEOUT
    # the hook was used up: the same call now succeeds and matches LAPACK
    lam, U = B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), 5)
    w = np.linalg.eigvalsh(G)[::-1]
    assert np.abs(lam.cpu().numpy() - w).max() <= 1e-12 * w[0]
    U = U.cpu().numpy()
    assert np.abs(U.T @ U - np.eye(5)).max() <= 1e-12


def test_htrise_update_that_times_out_leaves_the_state_unchanged(B):
    Y = S.gaussian_bumps(2, 0, 24)
    Y1, Y2 = Y[:8], Y[8:]          # the second batch expands the bases (a residual eigensolve runs)
    eps = 1e-4
    tree = B.bht_tree_create_balanced(Y.shape[1:])
    st = B.bht_l2r(tree, torch.from_numpy(Y1).cuda(), eps)
    ranks0 = B.bht_get_ranks(st)
    rec0 = B.ht_reconstruct(st, 0, 8, dtype="float64").cpu().numpy()
    cores0 = [B.bht_get_core(st, i) for i in range(1, len(ranks0))]
    B.bht_debug_withhold_barrier(1, 20)
    with pytest.raises(B.BHTError) as e:
        B.htrise_update(st, torch.from_numpy(Y2).cuda(), eps)
    assert e.value.status == BHT_ETIMEOUT
    assert B.bht_get_ranks(st) == ranks0
    assert np.array_equal(B.ht_reconstruct(st, 0, 8, dtype="float64").cpu().numpy(), rec0)
    for i, c0 in enumerate(cores0):
        assert np.array_equal(B.bht_get_core(st, i + 1), c0)
    # the same update again, now unhindered, equals an update of a fresh state
    info = B.htrise_update(st, torch.from_numpy(Y2).cuda(), eps)
    assert not info.skipped
    ref = B.bht_l2r(tree, torch.from_numpy(Y1).cuda(), eps)
    B.htrise_update(ref, torch.from_numpy(Y2).cuda(), eps)
    assert B.bht_get_ranks(st) == B.bht_get_ranks(ref)
    a = B.ht_reconstruct(st, 0, 24, dtype="float64").cpu().numpy()
    b = B.ht_reconstruct(ref, 0, 24, dtype="float64").cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(a - Y) <= eps * np.linalg.norm(Y) * (1 + 1e-9)
    B.bht_state_destroy(st)
    B.bht_state_destroy(ref)
    B.bht_tree_destroy(tree)

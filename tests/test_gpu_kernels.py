"""Kernel-level GPU checks through the C ABI: the node eigensolver against
LAPACK (numpy.linalg.eigh) and the tensor-core mode product against an FP64
matrix product, on shapes that span several tiles and ragged tails."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


@pytest.mark.parametrize("n", [1, 2, 3, 5, 33, 70, 96, 97, 130, 257, 961])
def test_sym_eig_matches_lapack(B, n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, n + 7)) * np.logspace(0, -6, n)[:, None]
    G = X @ X.T
    w = np.linalg.eigvalsh(G)[::-1]
    r = max(1, n // 2)
    lam, U = B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), r)
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    assert np.abs(lam - w).max() <= 1e-12 * w[0]
    assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-12
    resid = G @ U - U * lam[:r]
    assert np.abs(resid).max() <= 1e-10 * w[0]


# Vector counts and lengths that reach the other launch shapes of the blocked back-transformation:
# 8 vectors per CTA with more CTAs than SMs (1300 vectors), blocks of fewer than 16 reflectors next to
# them (1600 rows), and one vector alone.
@pytest.mark.parametrize("n,r", [(1600, 1300), (1600, 5)])
def test_sym_eig_many_vectors(B, n, r):
    rng = np.random.default_rng(n + r)
    X = rng.normal(size=(n, n + 7)) * np.logspace(0, -6, n)[:, None]
    G = X @ X.T
    w = np.linalg.eigvalsh(G)[::-1]
    lam, U = B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), r)
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    assert np.abs(lam - w).max() <= 1e-12 * w[0]
    assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-12
    resid = G @ U - U * lam[:r]
    assert np.abs(resid).max() <= 1e-10 * w[0]


# Every eigenvector of a Gram spectrum graded over twelve decades: its last 208 eigenvalues lie below
# 1e-9 ||G|| (one chain for the cluster Gram-Schmidt) with gaps down to 1.3e-15 ||G||. The inverse
# iteration spreads its shifts only along chains of numerically equal eigenvalues (gaps within
# 10 eps ||T||); spread over the whole 1e-9 chain they would move later members onto their neighbours.
def test_sym_eig_every_vector_of_graded_spectrum(B):
    n = r = 700
    rng = np.random.default_rng(n + r)
    X = rng.normal(size=(n, n + 7)) * np.logspace(0, -6, n)[:, None]
    G = X @ X.T
    w = np.linalg.eigvalsh(G)[::-1]
    lam, U = B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), r)
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    assert np.abs(lam - w).max() <= 1e-12 * w[0]
    assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-12
    resid = G @ U - U * lam[:r]
    assert np.abs(resid).max() <= 1e-10 * w[0]


def test_sym_eig_degenerate_pairs(B):
    rng = np.random.default_rng(3)
    n = 40
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    w = np.repeat(np.logspace(0, -4, n // 2), 2)          # every eigenvalue twice
    G = (Q * w) @ Q.T
    lam, U = B.bht_sym_eig(torch.from_numpy(G.copy()).cuda(), 10)
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    assert np.abs(lam - np.sort(w)[::-1]).max() <= 1e-12
    assert np.abs(U.T @ U - np.eye(10)).max() <= 1e-12
    # the span of the top 10 equals the span of the top 5 pairs
    P = Q[:, np.argsort(-w)[:10]]
    assert np.linalg.norm(U - P @ (P.T @ U), 2) <= 1e-8


@pytest.mark.parametrize("rows,K,S,R2", [(128, 64, 31, 1), (131072, 64, 31, 4096), (1000, 24, 7, 1),
                                         (333, 16, 16, 3), (4096, 96, 40, 64), (130, 4, 1, 1), (2048, 128, 128, 2)])
def test_tensor_core_mode_product(B, rows, K, S, R2):
    rng = np.random.default_rng(rows + K)
    X = rng.normal(size=(rows, K)).astype(np.float32)
    U = np.linalg.qr(rng.normal(size=(K, max(S, K))))[0][:, :S]
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    out = B.bht_mode_product(torch.from_numpy(X).cuda(), torch.from_numpy(np.ascontiguousarray(U)).cuda(), S,
                             "mixed", R2=R2, norms=norms).cpu().numpy().astype(np.float64)
    ref = X.astype(np.float64) @ U                       # [rows][S]
    o = rows // R2
    ref = ref.reshape(o, R2, S).transpose(0, 2, 1).reshape(-1)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 2e-5, err                               # split TF32, three products: about 2^-20 per product
    bias = (np.linalg.norm(out) ** 2 - np.linalg.norm(ref) ** 2) / np.linalg.norm(ref) ** 2
    assert abs(bias) < 1e-5, bias                        # no truncation or rounding bias in the norm
    n = norms.cpu().numpy()
    # ||X||^2: FP32 partial sums of 16 squares folded into FP64, so at most 16 * 2^-24 relative
    assert abs(n[0] - np.sum(X.astype(np.float64) ** 2)) <= 16 * 2.0 ** -24 * n[0]
    assert abs(n[1] - np.sum(out ** 2)) <= 1e-6 * n[1]


# The two-mode passes of small leaves on X [A][na][nb][B]: tiles of 32 columns of B (a ragged last block
# when B % 32 != 0, a single short block when B < 32), more tiles than SMs, FP32 products.
PAIR_SHAPES = [(5, 24, 24, 100), (7, 16, 9, 36), (2, 24, 7, 4), (300, 24, 24, 24), (3, 5, 24, 1000), (8, 24, 24, 13824)]


def _pair_input(A, na, nb, Bc, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(A, na, nb, Bc)) * np.linspace(1.0, 0.1, na)[None, :, None, None]
    return X.astype(np.float32)


@pytest.mark.parametrize("A,na,nb,Bc", PAIR_SHAPES)
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_pair_gram_matches_fp64(B, A, na, nb, Bc, tensor_cores):
    """24 x 24 pairs with tensor_cores take the split-TF32 tcgen05 pass; every other case the FP32 SIMT
    pass. The tensor-core pass accumulates one tile in FP32 in tensor memory: an entry receives 96 MMA
    results (24 row groups x 4 steps of 8 columns) per tile, each addition within 2^-23 of the partial
    sum, which bounds the error by 96 * 2^-23 < 1.2e-5 of the largest entry (the split products themselves
    are within 2^-22); the SIMT pass sums FP32 products per lane over at most a few hundred columns."""
    X = _pair_input(A, na, nb, Bc, A + na + nb)
    Ga, Gb = B.bht_pair_gram(torch.from_numpy(X).cuda(), tensor_cores=tensor_cores)
    X64 = X.astype(np.float64)
    Xa = X64.transpose(1, 0, 2, 3).reshape(na, -1)
    Xb = X64.transpose(2, 0, 1, 3).reshape(nb, -1)
    ra, rb = Xa @ Xa.T, Xb @ Xb.T
    Ga, Gb = Ga.cpu().numpy(), Gb.cpu().numpy()
    tol = 1.2e-5 if (tensor_cores and na == 24 and nb == 24) else 2e-6
    assert np.abs(Ga - ra).max() <= tol * np.abs(ra).max()
    assert np.abs(Gb - rb).max() <= tol * np.abs(rb).max()
    assert np.allclose(Ga, Ga.T, rtol=0, atol=1e-14 * np.abs(ra).max())
    assert np.allclose(Gb, Gb.T, rtol=0, atol=1e-14 * np.abs(rb).max())
    assert abs(np.trace(Ga) - np.sum(X64 ** 2)) <= max(tol, 1e-6) * np.sum(X64 ** 2)


@pytest.mark.parametrize("A,na,nb,Bc", PAIR_SHAPES)
@pytest.mark.parametrize("ra,rb", [(7, 7), (3, 16), (16, 1)])
def test_pair_project_matches_fp64(B, A, na, nb, Bc, ra, rb):
    ra, rb = min(ra, na), min(rb, nb)
    X = _pair_input(A, na, nb, Bc, A * 3 + ra)
    rng = np.random.default_rng(ra * 100 + rb)
    Ua = np.linalg.qr(rng.normal(size=(na, na)))[0][:, :ra].copy()
    Ub = np.linalg.qr(rng.normal(size=(nb, nb)))[0][:, :rb].copy()
    norms = torch.zeros(3, dtype=torch.float64, device="cuda")
    out = B.bht_pair_project(torch.from_numpy(X).cuda(), torch.from_numpy(Ua).cuda(), torch.from_numpy(Ub).cuda(),
                             norms=norms).cpu().numpy().astype(np.float64)
    ref = np.tensordot(np.tensordot(X.astype(np.float64), Ua, axes=([1], [0])), Ub, axes=([1], [0]))  # [A][B][ra][rb]
    ref = ref.transpose(0, 2, 3, 1)
    # FP32 products on FP32-rounded bases: about 2^-24 sqrt(na nb) relative
    assert np.linalg.norm(out - ref) <= 2e-6 * np.linalg.norm(ref)
    n = norms.cpu().numpy()
    x2, o2 = float(np.sum(X.astype(np.float64) ** 2)), float(np.sum(ref ** 2))
    assert abs(n[0] - x2) <= 1e-6 * x2
    assert abs(n[1] - o2) <= 2e-6 * o2
    assert abs(n[2] - (n[0] - n[1])) <= 1e-9 * x2


TRI_SHAPES = [
    (50, 24, 24, 24, 7, 7, 7),    # the 24^5 stream's last three leaves (one slab per item and column pair)
    (7, 24, 24, 24, 8, 1, 5),     # fewer slabs than SMs
    (300, 12, 20, 8, 3, 8, 2),    # ragged sizes, 300 slabs over the ring's three stages
    (5, 32, 16, 24, 8, 8, 8),     # a large slab (12288 values), ranks 8
    (1000, 1, 4, 1, 1, 2, 1),     # degenerate modes
]


@pytest.mark.parametrize("A,n1,n2,n3,r1,r2,r3", TRI_SHAPES)
def test_tri_project_matches_fp64(B, A, n1, n2, n3, r1, r2, r3):
    r1, r2, r3 = min(r1, n1), min(r2, n2), min(r3, n3)
    rng = np.random.default_rng(A + n1 + n2 + n3)
    X = (rng.normal(size=(A, n1, n2, n3)) * np.linspace(1.0, 0.1, n1)[None, :, None, None]).astype(np.float32)
    U = [np.linalg.qr(rng.normal(size=(n, n)))[0][:, :r].copy() for n, r in ((n1, r1), (n2, r2), (n3, r3))]
    norms = torch.zeros(3, dtype=torch.float64, device="cuda")
    out = B.bht_tri_project(torch.from_numpy(X).cuda(), *[torch.from_numpy(u).cuda() for u in U],
                            norms=norms).cpu().numpy().astype(np.float64)
    ref = np.einsum("xijk,ia,jb,kc->xabc", X.astype(np.float64), *U)
    # FP32 products on FP32-rounded bases, three contractions: about 2^-24 sqrt(n1 n2 n3) relative
    assert np.linalg.norm(out - ref) <= 4e-6 * np.linalg.norm(ref)
    n = norms.cpu().numpy()
    x2, o2 = float(np.sum(X.astype(np.float64) ** 2)), float(np.sum(ref ** 2))
    assert abs(n[0] - x2) <= 1e-6 * x2
    assert abs(n[1] - o2) <= 4e-6 * o2
    assert abs(n[2] - (n[0] - n[1])) <= 1e-9 * x2


def test_tri_project_arguments(B):
    X = torch.zeros((2, 24, 24, 24), dtype=torch.float32, device="cuda")
    U = torch.zeros((24, 7), dtype=torch.float64, device="cuda")
    for bad in [(2, 24, 24, 33, 7, 7, 7), (2, 24, 24, 24, 7, 9, 7), (2, 24, 3, 5, 7, 3, 5), (2, 32, 32, 32, 7, 7, 7)]:
        A, n1, n2, n3, r1, r2, r3 = bad
        st = B._lib.bht_tri_project(ctypes.c_void_p(X.data_ptr()), A, n1, n2, n3, ctypes.c_void_p(U.data_ptr()), r1,
                                    ctypes.c_void_p(U.data_ptr()), r2, ctypes.c_void_p(U.data_ptr()), r3,
                                    ctypes.c_void_p(X.data_ptr()), None, None)
        assert st == B.BHT_EUNSUPPORTED
    host = np.zeros(4, dtype=np.float32)
    st = B._lib.bht_tri_project(ctypes.c_void_p(host.ctypes.data), 1, 1, 4, 1, ctypes.c_void_p(U.data_ptr()), 1,
                                ctypes.c_void_p(U.data_ptr()), 1, ctypes.c_void_p(U.data_ptr()), 1,
                                ctypes.c_void_p(X.data_ptr()), None, None)
    assert st == B.BHT_EINVAL


def _small_gram(kind, n, rng):
    if kind == "graded":
        X = rng.normal(size=(n, n + 5)) * np.logspace(0, -4, n)[:, None]
    elif kind == "lowrank":
        X = rng.normal(size=(n, 3)) @ rng.normal(size=(3, 60)) + 1e-3 * rng.normal(size=(n, 60))
    elif kind == "random":
        X = rng.normal(size=(n, 2 * n))
    else:
        return np.zeros((n, n))
    return X @ X.T


@pytest.mark.parametrize("n", [1, 2, 7, 16, 17, 24, 31, 32])
@pytest.mark.parametrize("kind", ["graded", "lowrank", "random", "zero"])
def test_sym_eig_small_ritz_values(B, n, kind):
    """FP32 Jacobi vectors refined and made orthonormal in FP64, and their FP64 Ritz values: V is orthonormal to
    rounding, lam_i = v_i^T G v_i, and keeping the first r vectors discards sum_{i>=r} lam_i, which exceeds
    the optimal tail (the sum of the smallest eigenvalues) by at most the square of the vectors' FP32-level
    angles: 2e-7 of the trace allows for clusters inside the FP32 rounding of G (measured up to 5e-8)."""
    rng = np.random.default_rng(n * 7 + len(kind))
    G = _small_gram(kind, n, rng)
    lam, V = B.bht_sym_eig_small(torch.from_numpy(G).cuda())
    lam, V = lam.cpu().numpy(), V.cpu().numpy()
    tr = max(np.trace(G), 1e-300)
    assert np.all(np.diff(lam) <= 0)
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13
    assert np.abs(np.diag(V.T @ G @ V) - lam).max() <= 1e-12 * tr
    w, Ve = np.linalg.eigh(G)
    w, Ve = w[::-1], Ve[:, ::-1]
    for r in range(n):
        excess = lam[r:].sum() - w[r:].sum()
        assert -1e-12 * tr <= excess <= 2e-7 * tr
    # after the FP64 refinement, a split with a clear gap separates the kept and discarded spaces to
    # second order in the FP32 vectors' angles (about (1e-4)^2 without it at gaps of 1e-3 of the trace)
    for r in range(1, n):
        if w[r - 1] - w[r] > 1e-3 * tr:
            assert np.linalg.norm(Ve[:, :r].T @ V[:, r:], 2) <= 1e-6

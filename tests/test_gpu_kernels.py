"""Kernel-level GPU checks through the C ABI: the node eigensolver against
LAPACK (numpy.linalg.eigh) and the tensor-core mode product against an FP64
matrix product, on shapes that span several tiles and ragged tails."""
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

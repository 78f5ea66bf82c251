"""Data preparation kernels against the oracle: per-group normalisation (max-abs, unit vector, z-score,
Sec. 5.2) and its inverse, and the permutation of item axes (App. D axis orderings).

Normalisation: shift and scale are FP64 reductions of the same values on both sides, so they agree to
a few ulps (1e-13 relative); the normalised FP64 data to 1e-13, FP32 data to one FP32 rounding
(2^-23 relative) plus that. Permutation: a pure data movement, bit-exact.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["maxabs", "unitvec", "zscore", "none"])
@pytest.mark.parametrize("shape,groups", [((3, 5), 3), ((4, 2, 3 * 8192 + 17), 8), ((2, 5, 48, 48, 48), 10),
                                          ((7, 1000), 1)])
def test_normalize_matches_oracle(B, dtype, kind, shape, groups):
    rng = np.random.default_rng(len(shape) * 31 + groups)
    Y = (rng.normal(size=shape) * 3.0 + 1.5).astype(dtype)
    Yd = torch.from_numpy(Y.copy()).cuda()
    P = B.bht_normalize(Yd, kind, groups=groups)
    Yn, Po = O.normalize(Y, kind, groups=groups)
    assert np.allclose(P, Po, rtol=1e-13, atol=0)
    got = Yd.cpu().numpy().astype(np.float64)
    tol = 1e-13 if dtype == np.float64 else 2.0 ** -23
    assert np.all(np.abs(got - Yn) <= tol * np.abs(Yn) + 1e-13 * np.abs(Yn).max())
    B.bht_denormalize(Yd, P)
    back = Yd.cpu().numpy().astype(np.float64)
    tol = 1e-12 if dtype == np.float64 else 2.0 ** -21
    assert np.all(np.abs(back - Y) <= tol * np.abs(Y).max())


def test_normalize_constant_and_empty_groups(B):
    Yd = torch.full((3, 100), 2.5, device="cuda", dtype=torch.float64)
    P = B.bht_normalize(Yd, "zscore")
    assert np.array_equal(P[:, 1], np.ones(3)) and np.array_equal(P[:, 0], np.full(3, 2.5))
    assert float(Yd.abs().max()) == 0.0
    P0 = B.bht_normalize(torch.zeros((2, 0), device="cuda"), "maxabs", groups=2)
    assert P0.shape == (2, 2)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape,perm", [
    ((3, 7), [0]),
    ((2, 4, 6), [1, 0]),
    ((5, 3, 4, 5), [2, 0, 1]),
    ((2, 8, 8, 8, 8, 8, 8), [0, 1, 2, 5, 4, 3]),     # a transposition of two inner modes
    ((2, 8, 8, 8, 21, 8, 5), [0, 4, 2, 3, 1, 5]),
    ((1, 2, 3, 4, 5, 6, 7), [5, 4, 3, 2, 1, 0]),
])
def test_permute_items_is_numpy_transpose(B, dtype, shape, perm):
    X = torch.randn(shape, dtype=dtype, device="cuda")
    out = B.bht_permute_items(X, perm)
    want = np.transpose(X.cpu().numpy(), [0] + [1 + p for p in perm])
    assert out.shape == want.shape
    assert np.array_equal(out.cpu().numpy(), want)


def test_permute_items_rejects_bad_input(B):
    X = torch.randn((2, 3, 4), device="cuda")
    with pytest.raises(B.BHTError):
        B.bht_permute_items(X, [0, 0])
    with pytest.raises(ValueError):
        B.bht_permute_items(X, [0])

"""bht_mode_product_noalloc against bht_mode_product, through the C ABI.

The no-allocation entry point serves callers that may not allocate device
memory during a call (their memory is owned by another allocator, or the call
sits in a latency-critical loop). It must give the same product as the
allocating entry point, twice in a row (its static scratch keeps the previous
call's contents), and refuse sizes beyond its static scratch. This file is
collected last on purpose.
"""
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


def test_noalloc_matches_allocating_entry_point_twice(B):
    cases = [(131072, 64, 31, 4096, 1), (3000, 24, 7, 1, 2)]  # two calls in a row, different shapes
    for rows, K, S, R2, seed in cases:
        rng = np.random.default_rng(seed)
        X = torch.from_numpy(rng.normal(size=(rows, K)).astype(np.float32)).cuda()
        U = torch.from_numpy(np.ascontiguousarray(np.linalg.qr(rng.normal(size=(K, K)))[0][:, :S])).cuda()
        ref = B.bht_mode_product(X, U, S, "mixed", R2=R2)
        out = torch.full((rows * S,), float("nan"), dtype=torch.float32, device="cuda")
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        B.bht_mode_product_noalloc(X, U, S, R2=R2, out=out, norms=norms)
        torch.cuda.synchronize()
        a, b = out.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= 2e-5 * np.linalg.norm(b)
        n = norms.cpu().numpy()
        # ||X||^2 from FP32 partial sums of 16 squares folded into FP64: at most 16 * 2^-24 relative
        assert abs(n[0] - float(torch.sum(X.double() ** 2))) <= 16 * 2.0 ** -24 * n[0]


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    X = torch.zeros((128, 1024), dtype=torch.float32, device="cuda")
    U = torch.zeros((1024, 8), dtype=torch.float64, device="cuda")
    out = torch.zeros(128 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(B.BHTError) as e:
        B.bht_mode_product_noalloc(X, U, 8, out=out)
    assert e.value.status == 3  # BHT_ECAPACITY

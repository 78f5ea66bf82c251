"""The format studies (BHT vs plain HT, tensorisation, axis order, normalisation) at small sizes: every
configuration runs through the library and reports finite, consistent figures."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_16544_gb300 import sweeps
    return sweeps


def test_bht_vs_ht_small(W):
    rows = W.bht_vs_ht(grid=32, batches=(8, 16), eps_list=(0.1,), norms=("none", "zscore"))
    assert len(rows) == 4
    for r in rows:
        assert r["bht_cr"] > 1.0 and r["ht_cr"] > 1.0
        assert r["bht_ms"] > 0 and r["ht_ms"] > 0
        assert r["ht_ranks"][0] == 1 and r["bht_ranks"][0] == r["N"]


def test_reshape_axis_order_normalize_small(W):
    rows = W.reshape(grid=16, items=16, inc=8, test=4) + W.axis_order(items=16, inc=8, test=4) + \
        W.normalize(grid=16, items=16, inc=8, test=4) + W.budget(grid=16, items=16, inc=8, test=4, eps_list=(1e-1,))
    assert len(rows) == 2 + 4 + 4 + 2
    for r in rows:
        assert "failed" not in r, r
        assert r["cr"] > 0 and r["rr"] >= 1.0 and math.isfinite(r["rte"]) and 0 <= r["rte"] < 1


def test_adaptive_budget_keeps_the_per_increment_bound(W):
    rows = W.budget(grid=32, items=32, inc=16, test=4, eps_list=(1e-1,))
    uni, ada = rows
    assert uni["budget"] == "uniform" and ada["budget"] == "adaptive"
    assert ada["max_err_over_eps"] <= 1.0 + 1e-4 and uni["max_err_over_eps"] <= 1.0 + 1e-4

"""The seeded input generators on the CPU: the counter-based normals are standard normal and
independent across items and seeds, and a stream's items can be regenerated one at a time."""
import numpy as np
import pytest

import bht_synth as S

scipy_stats = pytest.importorskip("scipy.stats")


def test_counter_normals_are_standard_normal():
    z = np.concatenate([S.counter_normals(s, m, 200_000) for s in (0, 1) for m in (0, 1, 2)])
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.std() - 1.0) < 5 / np.sqrt(2 * z.size)
    assert scipy_stats.kstest(z, "norm").pvalue > 1e-4
    # the cosine and sine halves of a word are uncorrelated, as are neighbouring items
    a = S.counter_normals(0, 0, 400_000)
    assert abs(np.corrcoef(a[0::2], a[1::2])[0, 1]) < 5 / np.sqrt(200_000)
    b = S.counter_normals(0, 1, 400_000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(400_000)


def test_counter_normals_prefix_and_item_independence():
    a = S.counter_normals(3, 17, 1001)
    assert np.array_equal(a[:500], S.counter_normals(3, 17, 500))
    assert not np.allclose(a, S.counter_normals(3, 18, 1001))
    assert not np.allclose(a, S.counter_normals(4, 17, 1001))


def test_mix64_is_the_splitmix64_output_function():
    # the first outputs of SplitMix64 seeded with 0 (the sequence mix64(k * gamma), k = 1, 2, ...)
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        w = S._mix64(np.arange(1, 4, dtype=np.uint64) * g)
    assert [int(x) for x in w] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sensor_items_regenerate_one_at_a_time():
    Y = S.chebyshev_sensor(2, 5, 3, n=8, d=3)
    for j in range(3):
        assert np.array_equal(Y[j], S.chebyshev_sensor(2, 5 + j, 1, n=8, d=3)[0])

"""The device generator of the Chebyshev sensor stream against bht_synth.chebyshev_sensor, item by item.

Both sides draw the same coefficients (numpy, per item) and the same counter-based normals; the device
sums the separable products and the Box-Muller transform in FP32, the host in FP64 (then rounds to
fp32). The tolerance is 1e-5 of the item's largest magnitude: 20 terms of FP32 products and sums carry
about 20 * 2^-24 relative error each.
"""
import numpy as np
import pytest

import bht_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


@pytest.mark.parametrize("n,d,first,count,noise", [(24, 5, 0, 2, 0.01), (24, 5, 3137, 1, 0.01),
                                                    (12, 4, 5, 8, 0.01), (7, 3, 0, 5, 0.5), (10, 2, 2, 3, 0.0),
                                                    (24, 5, 64, 2, 0.0)])
def test_device_generator_matches_host(B, n, d, first, count, noise):
    c = S.chebyshev_coefficients(0, first, count, d=d)
    dev = B.bht_synth_chebyshev(c, n, seed=0, first_item=first, noise_std=noise).cpu().numpy()
    host = S.chebyshev_sensor(0, first, count, n=n, d=d, noise_std=noise)
    for j in range(count):
        scale = np.abs(host[j]).max()
        assert np.abs(dev[j] - host[j]).max() <= 1e-5 * scale, j


def test_device_generator_from_device_coefficients_and_seed(B):
    c = S.chebyshev_coefficients(7, 10, 3, d=4)
    a = B.bht_synth_chebyshev(torch.from_numpy(c).cuda(), 12, seed=7, first_item=10).cpu().numpy()
    b = S.chebyshev_sensor(7, 10, 3, n=12, d=4)
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    # another seed draws other noise from the same coefficients
    o = B.bht_synth_chebyshev(c, 12, seed=8, first_item=10).cpu().numpy()
    assert np.abs(o - a).max() > 1e-3


def test_device_generator_rejects_bad_arguments(B):
    c = S.chebyshev_coefficients(0, 0, 1, d=3)
    with pytest.raises(B.BHTError):
        B.bht_synth_chebyshev(c, 65, seed=0, first_item=0)        # n beyond 64
    with pytest.raises(B.BHTError):
        B.bht_synth_chebyshev(c, 8, seed=0, first_item=-1)        # negative first item

"""bht_mode_product_noalloc against bht_mode_product, through the C ABI.

The no-allocation entry point serves callers that may not allocate device
memory during a call (their memory is owned by another allocator, or the call
sits in a latency-critical loop). It must give the same product as the
allocating entry point, twice in a row (its static scratch keeps the previous
call's contents), allocate nothing (neither the device's free memory nor the
stream-ordered pool's use moves during a call), and refuse sizes beyond its
static scratch and host pointers with error codes. This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_POOL_USED_CURRENT, _POOL_USED_HIGH = 7, 8   # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH (cuda.h)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


class PoolWatch:
    """Use of the device's default stream-ordered pool, through the driver API: the high-water mark is
    reset before a call and read after it, so an allocation freed inside the call still shows."""

    def __init__(self):
        cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0
        self.cu = cu

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, _POOL_USED_HIGH, ctypes.byref(z)) == 0


def test_noalloc_matches_allocating_entry_point_twice(B):
    watch = PoolWatch()
    cases = [(131072, 64, 31, 4096, 1), (3000, 24, 7, 1, 2)]  # two calls in a row, different shapes
    for rows, K, S, R2, seed in cases:
        rng = np.random.default_rng(seed)
        X = torch.from_numpy(rng.normal(size=(rows, K)).astype(np.float32)).cuda()
        U = torch.from_numpy(np.ascontiguousarray(np.linalg.qr(rng.normal(size=(K, K)))[0][:, :S])).cuda()
        ref = B.bht_mode_product(X, U, S, "mixed", R2=R2)
        out = torch.full((rows * S,), float("nan"), dtype=torch.float32, device="cuda")
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        used0 = watch.get(_POOL_USED_CURRENT)
        watch.reset_high()
        B.bht_mode_product_noalloc(X, U, S, R2=R2, out=out, norms=norms)
        torch.cuda.synchronize()
        assert watch.get(_POOL_USED_HIGH) <= used0      # no stream-ordered allocation, not even a freed one
        assert torch.cuda.mem_get_info()[0] == free0    # no device memory taken and kept
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


def test_noalloc_rejects_host_pointers(B):
    """A host buffer is refused by the library's pointer check before anything is launched."""
    Xh = np.zeros((256, 16), dtype=np.float32)
    U = torch.zeros((16, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(256 * 4, dtype=torch.float32, device="cuda")
    st = B.lib().bht_mode_product_noalloc(ctypes.c_void_p(Xh.ctypes.data), 256, 16, ctypes.c_void_p(U.data_ptr()),
                                          4, ctypes.c_void_p(out.data_ptr()), 1, None, None)
    assert st == 1  # BHT_EINVAL
    with pytest.raises(ValueError):
        B.bht_mode_product_noalloc(torch.from_numpy(Xh), U, 4, out=out)

"""htrise_update_stream against the same batches fed one by one to htrise_update.

The stream entry enqueues Step 1 of batch k + 1 before it reads back the skip test of batch k, and
fills device buffers from host batches on a copy stream. Its result must be that of Algorithm 2 run
batch by batch: the same skip decisions and projection errors, the same ranks and item count, and the
same decoded items up to the order of the floating-point reductions (atomic FP64 sums).

* the graded two-way stream at eps = 1e-6 (FP64): the first update expands the leaf, so the
  speculative projection of the next batch is dropped and made again, and the last batch is skipped;
* the Chebyshev sensor stream at 12^4 (mixed): batches from device memory, pinned host memory and
  pageable host memory, skips throughout.
"""
import ctypes

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


def _compare(B, sa, sb, infos_a, infos_b, rtol, dtype):
    """Same decisions and ranks; decoded items within rtol ||Y_items|| (cores inside clusters of nearly
    equal eigenvalues are not unique, so they are compared through what they decode to)."""
    assert [i.skipped for i in infos_a] == [i.skipped for i in infos_b]
    for ia, ib in zip(infos_a, infos_b):
        # the FP64 form takes the error as ||Y||^2 - ||C||^2: compare its square against ||Y||^2
        assert abs(ib.eps_proj ** 2 - ia.eps_proj ** 2) <= max(rtol * ia.eps_proj ** 2, 1e-13 * ia.norm_y ** 2)
        assert ib.norm_y == pytest.approx(ia.norm_y, rel=1e-12)
        assert ib.eps_des == pytest.approx(ia.eps_des, rel=1e-12)
        assert ib.n_items_total == ia.n_items_total
        assert ib.batch_reads == ia.batch_reads
    assert B.bht_get_ranks(sa) == B.bht_get_ranks(sb)
    n = infos_a[-1].n_items_total
    ya = B.ht_reconstruct(sa, 0, n, dtype=dtype).double()
    yb = B.ht_reconstruct(sb, 0, n, dtype=dtype).double()
    assert float(torch.linalg.vector_norm(ya - yb)) <= rtol * float(torch.linalg.vector_norm(ya))


def test_stream_graded_expand_then_skip(B):
    batches = S.graded_stream(0)
    eps = 1e-6
    tree = B.bht_tree_create_balanced([400, 6])
    Y0 = torch.from_numpy(batches[0]).cuda()
    rest = torch.from_numpy(np.stack(batches[1:])).cuda()   # [2][48][400][6]
    sa = B.bht_l2r(tree, Y0, eps, precision="fp64")
    sb = B.bht_l2r(tree, Y0, eps, precision="fp64")
    infos_a = [B.htrise_update(sa, rest[k], eps, precision="fp64") for k in range(rest.shape[0])]
    infos_b = B.htrise_update_stream(sb, rest, eps, precision="fp64")
    assert [i.skipped for i in infos_b] == [False, True]
    _compare(B, sa, sb, infos_a, infos_b, 1e-9, "float64")
    B.bht_state_destroy(sa)
    B.bht_state_destroy(sb)


@pytest.mark.parametrize("where", ["device", "pinned", "pageable"])
def test_stream_sensor_sources(B, where):
    eps = 1e-2
    n, d, per, count = 12, 4, 8, 5
    Y = S.chebyshev_sensor(0, 0, per * (count + 1), n=n, d=d).astype(np.float32)
    Y = Y.reshape(count + 1, per, *([n] * d))
    tree = B.bht_tree_create_balanced([n] * d)
    Yd = torch.from_numpy(Y).cuda()
    sa = B.bht_l2r(tree, Yd[0], eps, precision="mixed")
    sb = B.bht_l2r(tree, Yd[0], eps, precision="mixed")
    infos_a = [B.htrise_update(sa, Yd[k], eps, precision="mixed") for k in range(1, count + 1)]
    if where == "device":
        src = Yd[1:]
    elif where == "pinned":
        src = torch.from_numpy(Y[1:].copy()).pin_memory()
    else:
        src = np.ascontiguousarray(Y[1:])
    infos_b = B.htrise_update_stream(sb, src, eps, precision="mixed")
    _compare(B, sa, sb, infos_a, infos_b, 1e-5, "float32")
    assert infos_b[-1].n_items_total == per * (count + 1)
    B.bht_state_destroy(sa)
    B.bht_state_destroy(sb)


def test_stream_arguments(B):
    eps = 1e-2
    Y = S.chebyshev_sensor(0, 0, 8, n=8, d=3).astype(np.float32)
    tree = B.bht_tree_create_balanced([8] * 3)
    Yd = torch.from_numpy(Y).cuda()
    st = B.bht_l2r(tree, Yd[:4], eps, precision="mixed")
    done = ctypes.c_int64(-1)
    lib = B._lib
    # zero batches: nothing happens
    assert lib.htrise_update_stream(st, ctypes.c_void_p(Yd.data_ptr()), B.BHT_F32, 4, 0, eps, None, None, None,
                                    ctypes.byref(done)) == B.BHT_OK
    assert done.value == 0
    # bad arguments are refused before any work
    assert lib.htrise_update_stream(st, ctypes.c_void_p(Yd.data_ptr()), B.BHT_F32, 0, 1, eps, None, None, None,
                                    ctypes.byref(done)) == B.BHT_EINVAL
    assert lib.htrise_update_stream(st, ctypes.c_void_p(Yd.data_ptr()), B.BHT_F32, 4, -1, eps, None, None, None,
                                    ctypes.byref(done)) == B.BHT_EINVAL
    assert lib.htrise_update_stream(st, ctypes.c_void_p(Yd.data_ptr()), B.BHT_F32, 4, 1, -1.0, None, None, None,
                                    ctypes.byref(done)) == B.BHT_EINVAL
    assert lib.htrise_update_stream(st, None, B.BHT_F32, 4, 1, eps, None, None, None,
                                    ctypes.byref(done)) == B.BHT_EINVAL
    # one batch through the stream entry, then the state is still usable by htrise_update
    infos = B.htrise_update_stream(st, Yd[4:].reshape(1, 4, 8, 8, 8), eps, precision="mixed")
    assert len(infos) == 1 and infos[0].n_items_total == 8
    B.bht_state_destroy(st)

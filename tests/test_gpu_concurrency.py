"""Independent streams compressed concurrently, one host thread and one CUDA stream each, against the
same streams compressed one after another, through the C ABI.

The library's process-wide state (the stream-ordered pool, the cached tensor-core weight planes of
committed cores, the shared-memory limits raised per kernel, the profiler and the launch counters) is
shared by the threads. Results must not depend on the interleaving: the ranks are equal and the
reconstructions agree to the run-to-run rounding of the FP64 atomic sums in the Gram kernels.
"""
import threading

import numpy as np
import pytest

import bht_synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STREAMS = 6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2412_16544_gb300 as B
    return B


def _stream_data(sidx):
    if sidx % 2 == 0:
        Y = S.spectral_field(sidx, 0, 24, n=32)                      # 32^3, increments of 8
        return [torch.from_numpy(Y[k:k + 8]).cuda() for k in (0, 8, 16)], 1e-2
    sizes = [int(x) for x in S.increment_sizes(sidx, 3, 1, 12)]     # 5 x 16^3, uneven increments
    Y = torch.from_numpy(S.multivar_field(sidx, 0, sum(sizes), n=16)).cuda()
    return list(torch.split(Y, sizes)), 1e-3


def _compress(B, tree_of, batches, eps, precision, cs, out, i):
    try:
        with torch.cuda.stream(cs):
            tree = tree_of(batches[0].shape[1:])
            st = B.bht_l2r(tree, batches[0], eps, precision=precision, stream=cs)
            for Yk in batches[1:]:
                B.htrise_update(st, Yk, eps, precision=precision, stream=cs)
            cs.synchronize()
            out[i] = st
    except Exception as e:  # reported by the main thread
        out[i] = e


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_concurrent_streams_equal_sequential(B, precision):
    data = [_stream_data(i) for i in range(STREAMS)]
    trees = {}
    lock = threading.Lock()

    def tree_of(dims):
        with lock:
            key = tuple(dims)
            if key not in trees:
                trees[key] = B.bht_tree_create_balanced(list(dims))
            return trees[key]

    def run(concurrent):
        out = [None] * STREAMS
        if concurrent:
            cs = [torch.cuda.Stream() for _ in range(STREAMS)]
            th = [threading.Thread(target=_compress, args=(B, tree_of, data[i][0], data[i][1], precision, cs[i], out, i))
                  for i in range(STREAMS)]
            for t in th:
                t.start()
            for t in th:
                t.join()
        else:
            cs = torch.cuda.current_stream()
            for i in range(STREAMS):
                _compress(B, tree_of, data[i][0], data[i][1], precision, cs, out, i)
        torch.cuda.synchronize()
        for x in out:
            if isinstance(x, Exception):
                raise x
        return out

    seq = run(False)
    for rep in range(2):
        conc = run(True)
        for i in range(STREAMS):
            assert B.bht_get_ranks(conc[i]) == B.bht_get_ranks(seq[i]), (i, rep)
            n = B.bht_get_ranks(seq[i])[0]
            a = B.ht_reconstruct(seq[i], 0, n, dtype="float64")
            b = B.ht_reconstruct(conc[i], 0, n, dtype="float64")
            d = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a))
            assert d <= 1e-9, (i, rep, d)
            Yall = torch.cat([y.double() for y in data[i][0]])
            assert float(torch.linalg.vector_norm(b - Yall)) <= data[i][1] * float(torch.linalg.vector_norm(Yall)) * 1.0001
        for x in conc:
            B.bht_state_destroy(x)
    for x in seq:
        B.bht_state_destroy(x)
    for t in trees.values():
        B.bht_tree_destroy(t)

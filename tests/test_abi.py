"""The C-ABI library loads, exports every entry point of include/bht.h, and its
host-only logic (tree construction, argument checks) behaves on a machine
without a GPU. No call here touches the device."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:bht_status|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def bht():
    import paper_2412_16544_gb300 as B
    return B


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for n in ("bht_l2r", "htrise_update", "ht_reconstruct", "ht_encode", "bht_tree_create_balanced",
              "bht_state_destroy", "bht_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(bht):
    out = subprocess.run(["nm", "-D", "--defined-only", bht.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(bht.lib(), n)
        assert n in bht.EXPORTED


def test_library_has_no_oracle_or_python_dependency(bht):
    out = subprocess.run(["nm", "-D", bht.LIB_PATH], capture_output=True, text=True).stdout
    assert "Py" not in re.findall(r" U (\w+)", out)
    libs = subprocess.run(["ldd", bht.LIB_PATH], capture_output=True, text=True).stdout
    assert "python" not in libs and "torch" not in libs


@pytest.mark.parametrize("d", [2, 3, 4, 5, 7, 8, 16])
def test_tree_depth_host_only(bht, d):
    t = bht.bht_tree_create_balanced([5] * d)
    depth, nodes = bht.bht_tree_info(t)
    bht.bht_tree_destroy(t)
    assert depth == math.ceil(math.log2(d))
    assert nodes == 2 * d - 1


@pytest.mark.parametrize("dims", [[5], [], [3, 0, 4], [2] * 17, [5000, 2]])
def test_tree_rejects_bad_sizes(bht, dims):
    with pytest.raises(bht.BHTError) as e:
        bht.bht_tree_create_balanced(dims)
    assert e.value.status == 1  # BHT_EINVAL


def test_null_arguments_are_rejected(bht):
    L = bht.lib()
    assert L.bht_l2r(None, None, 0, 1, 0.1, None, None, None) == 1
    assert L.htrise_update(None, None, 0, 1, 0.1, None, None, None) == 1
    assert L.ht_reconstruct(None, 0, 1, None, 0, None) == 1
    assert L.bht_get_ranks(None, None, 0) == 1
    assert L.bht_state_destroy(None) == 0
    assert bht.bht_version().startswith("bht-gb300")


def test_eps_and_size_checks_before_any_device_work(bht):
    L = bht.lib()
    t = bht.bht_tree_create_balanced([4, 4])
    out = ctypes.c_void_p()
    buf = (ctypes.c_float * 16)()
    assert L.bht_l2r(t, buf, 0, 1, -1.0, None, None, ctypes.byref(out)) == 1      # eps <= 0
    assert L.bht_l2r(t, buf, 0, 0, 0.1, None, None, ctypes.byref(out)) == 1       # N = 0
    assert L.bht_l2r(t, buf, 7, 1, 0.1, None, None, ctypes.byref(out)) == 1       # dtype
    bht.bht_tree_destroy(t)


def test_sweep_tensorisations_keep_the_snapshot_size():
    import numpy as np
    from paper_2412_16544_gb300 import sweeps as W
    for g in (4, 16, 64):
        for name, shape in W.reshapes(g).items():
            assert int(np.prod(shape)) == g ** 3 and len(shape) <= 16, name
    for name, perm in W.AXIS_ORDERS.items():
        assert sorted(perm) == list(range(6)), name


def test_kernel_source_hash_follows_the_kernel_text_only():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    h = m.kernel_source_hash("eig_tridiag_f64")
    assert h is not None and len(h) == 64
    assert m.kernel_source_hash("no_such_class") is None
    src = open(os.path.join(ROOT, "paper_2412_16544_gb300", "csrc", "eig.cu")).read()
    body = m.function_text(src, "tridiag_rows_kernel")
    assert body.lstrip().startswith("__global__") and body.rstrip().endswith("}")
    assert body.count("{") == body.count("}")

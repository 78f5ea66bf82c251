"""Plain FP64 CPU oracle for BHT-l2r and HT-RISE (test infrastructure only).

This package is the checker, not the product. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. The GPU library never imports, links or calls anything here, and nothing
here imports the GPU library: the two share no code.

Everything is NumPy in float64, with SVDs of explicit unfoldings, following
the paper's algorithms step by step (see ``bht_oracle``).
"""
from .bht_oracle import (  # noqa: F401
    Tree, Node, dimension_tree, truncation_rank, truncated_left_svd,
    BHTState, UpdateInfo, bht_l2r, htrise_update, project, reconstruct, decode, relative_test_error,
    ht_l2r, ht_items, reduction_ratio, normalize,
    compression_ratio, layer_shape,
)
from . import mlp_oracle  # noqa: F401

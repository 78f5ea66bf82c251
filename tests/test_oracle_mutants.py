"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch each one.

A mutant that every pin accepts would mean the pins cannot tell a broken
oracle from a correct one.
"""
import types

import numpy as np
import pytest

import oracle.bht_oracle as B
import test_oracle_pins as P

PINS = [
    P.test_truncation_rank_brute_force,
    P.test_tiny_brute_force_ranks_and_root,
    P.test_exact_recovery_known_ranks_d5,
    lambda: P.test_d2_single_item_is_truncated_svd(0.05),
    P.test_d2_batch_is_truncated_hosvd,
    lambda: P.test_bht_error_bound_and_norm_identity((5, 4, 6), 0.1),
    lambda: P.test_bht_error_bound_and_norm_identity((3, 3, 4, 3, 3), 0.3),
    P.test_nodewise_errors_sum_bound,
    P.test_htrise_bound_invariance_orthonormality_c0,
    P.test_skip_projection_norm_identity,
    P.test_incremental_equals_one_shot_when_first_batch_spans,
    P.test_known_rank_growth,
]


def caught() -> bool:
    for pin in PINS:
        try:
            pin()
        except Exception:
            return True
    return False


def _no_sqrt_constant():
    fake = types.SimpleNamespace(sqrt=lambda x: 1.0)
    return ("math", fake)


def _rank_minus_one():
    orig = B.truncation_rank

    def bad(s2, eps_nw2, rmin):
        return max(orig(s2, eps_nw2, rmin) - 1, rmin)
    return ("truncation_rank", bad)


def _rank_strict_less():
    def bad(s2, eps_nw2, rmin):
        s2 = np.asarray(s2, dtype=np.float64)
        tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])
        ok = np.nonzero(tail < eps_nw2)[0]
        r = int(ok[0]) if len(ok) else len(s2)
        return min(max(r, rmin), len(s2))
    return ("truncation_rank", bad)


def _fortran_merge():
    orig = B._reshape_to_layer

    def bad(tree, C, axes, layer):
        out, new_axes = orig(tree, C, axes, layer)
        # merge transfer axes in Fortran order instead of C-order
        pos, arrs = 0, C
        shape = []
        for nd in tree.layer_nodes(layer):
            if nd.is_leaf:
                shape.append(arrs.shape[pos]); pos += 1
            else:
                arrs = np.swapaxes(arrs, pos, pos + 1)
                shape.append(arrs.shape[pos] * arrs.shape[pos + 1]); pos += 2
        return arrs.reshape(shape + [arrs.shape[-1]]), new_axes
    return ("_reshape_to_layer", bad)


def _pad_in_front():
    def bad(A, axis, extra):
        if extra == 0:
            return A
        shape = list(A.shape)
        shape[axis] = extra
        return np.concatenate([np.zeros(shape, dtype=A.dtype), A], axis=axis)
    return ("_pad_axis", bad)


def _transposed_projection():
    def bad(C, axis, U):
        if U.shape[0] == U.shape[1]:
            U = U.T
        else:
            U = U[::-1]  # rows permuted: a wrong index into the basis
        out = np.tensordot(C, U, axes=([axis], [0]))
        return np.moveaxis(out, -1, axis)
    return ("mode_product_t", bad)


def _no_reorthogonalisation_and_no_residual_projection():
    def bad(U_R, U_old):
        return U_R
    orig_svd = B.truncated_left_svd

    def bad_svd(M, eps_nw, rmin=1):
        return orig_svd(M, eps_nw * 3.0, rmin)
    return [("_orthogonalize_against", bad), ("truncated_left_svd", bad_svd)]


MUTANTS = {
    "no sqrt(2d-2) in eps_nw": _no_sqrt_constant,
    "rank off by one": _rank_minus_one,
    "strict < in tail rule": _rank_strict_less,
    "Fortran-order merge": _fortran_merge,
    "zero padding prepended": _pad_in_front,
    "projection with permuted basis": _transposed_projection,
    "node tolerance 3x too loose": _no_reorthogonalisation_and_no_residual_projection,
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    patches = MUTANTS[name]()
    if isinstance(patches, tuple):
        patches = [patches]
    for attr, val in patches:
        monkeypatch.setattr(B, attr, val)
    assert caught(), f"no pin failed for mutant: {name}"

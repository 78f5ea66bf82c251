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
    # the "next" rows: adaptive budget, decode / relative test error, normalisations, plain HT
    P.test_adaptive_budget_tolerance_formula,
    P.test_adaptive_budget_truncates_the_upper_layer_at_least_as_hard,
    P.test_decode_of_a_unit_latent_by_explicit_loops,
    P.test_decode_is_an_isometry_and_the_adjoint_of_projection,
    P.test_relative_test_error_closed_forms,
    P.test_reduction_ratio_and_normalisations,
    P.test_plain_ht_two_mode_items_are_the_truncated_svd_of_the_matricisation,
    P.test_plain_ht_recovers_known_ranks,
]


def _plain_ht_tolerance_pin():
    with pytest.MonkeyPatch.context() as mp:
        P.test_plain_ht_error_bound_and_tolerance(mp, 0.1)


PINS.append(_plain_ht_tolerance_pin)


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


def _plain_ht_uniform_constant():
    # the BHT constant sqrt(2(d+1) - 2) in place of the HT one sqrt(2(d+1) - 3)
    orig = B.ht_l2r

    def bad(Y, eps_rel):
        d1 = np.asarray(Y).ndim  # d + 1 modes, batch included
        return orig(Y, eps_rel * np.sqrt(2 * d1 - 3) / np.sqrt(2 * d1 - 2))
    return ("ht_l2r", bad)


def _decode_children_swapped():
    def bad(state, Z):
        tree = state.tree
        C = np.moveaxis(np.asarray(Z, dtype=np.float64), 0, -1)
        tags = list(tree.nodes[0].children)
        for layer in range(1, tree.p + 1):
            for nd in tree.layer_nodes(layer):
                ax = tags.index(nd.id)
                G = state.cores[nd.id]
                if nd.is_leaf:
                    C = np.moveaxis(np.tensordot(C, G, axes=([ax], [1])), -1, ax)
                    tags[ax] = ("mode", nd.mode)
                else:
                    out = np.tensordot(C, G, axes=([ax], [2]))
                    C = np.moveaxis(out, [-1, -2], [ax, ax + 1])   # children in the wrong order
                    tags[ax:ax + 1] = list(nd.children)
        return np.moveaxis(C, -1, 0)
    return ("decode", bad)


def _rte_aggregate():
    def bad(state, X, per_item=False):
        X = np.asarray(X, dtype=np.float64)
        e = float(np.linalg.norm(X - B.decode(state, B.project(state, X))) / np.linalg.norm(X))
        return (e, np.full(X.shape[0], e)) if per_item else e
    return ("relative_test_error", bad)


def _zscore_sample_std():
    orig = B.normalize

    def bad(Y, kind, groups=None):
        if kind != "zscore":
            return orig(Y, kind, groups)
        Y = np.asarray(Y, dtype=np.float64)
        groups = Y.shape[0] if groups is None else groups
        G = Y.reshape(groups, -1)
        mu, sd = G.mean(axis=1), G.std(axis=1, ddof=1)
        sd = np.where(sd > 0, sd, 1.0)
        return ((G - mu[:, None]) / sd[:, None]).reshape(Y.shape), np.column_stack([mu, sd])
    return ("normalize", bad)


def _adaptive_ignores_spent_error():
    def bad(eps_abs2, norm2, C, svd_rem):
        return float(np.sqrt(eps_abs2 / svd_rem))
    return ("_adaptive_eps_nw", bad)


MUTANTS = {
    "no sqrt(2d-2) in eps_nw": _no_sqrt_constant,
    "rank off by one": _rank_minus_one,
    "strict < in tail rule": _rank_strict_less,
    "Fortran-order merge": _fortran_merge,
    "zero padding prepended": _pad_in_front,
    "projection with permuted basis": _transposed_projection,
    "node tolerance 3x too loose": _no_reorthogonalisation_and_no_residual_projection,
    "plain HT with the BHT tolerance constant": _plain_ht_uniform_constant,
    "decode with a transfer core's children swapped": _decode_children_swapped,
    "relative test error as one aggregate ratio": _rte_aggregate,
    "z-score with the sample standard deviation": _zscore_sample_std,
    "adaptive budget ignoring the error already spent": _adaptive_ignores_spent_error,
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    patches = MUTANTS[name]()
    if isinstance(patches, tuple):
        patches = [patches]
    import oracle
    for attr, val in patches:
        monkeypatch.setattr(B, attr, val)
        if hasattr(oracle, attr):  # the package re-exports some names: patch what the pins call
            monkeypatch.setattr(oracle, attr, val)
    assert caught(), f"no pin failed for mutant: {name}"

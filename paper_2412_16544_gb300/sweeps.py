"""Studies of the format on synthetic data, driven through the library's calls.

* ``bht_vs_ht``   one-shot BHT-l2r against the plain HT leaves-to-root baseline (batch as the last leaf)
                  over batch sizes, tolerances and normalisations: compression ratio and time (App. D.1).
* ``reshape``     the same snapshots tensorised with different item shapes (64^3 as 8^6, 4^9, ...),
                  compressed as a stream with BHT-l2r + HT-RISE: time, CR, RR, RTE (App. D.2).
* ``axis_order``  item axes permuted on the GPU before the stream (App. D.3).
* ``normalize``   the multi-variable stream with each physical quantity of each snapshot normalised on
                  its own (none, max-abs, unit vector, z-score; Sec. 5.2): time, CR, RR, RTE.
* ``budget``      the uniform node-wise tolerance against the adaptive budget of App. C.

The snapshots are the advected spectral fields of ``bht_synth`` (stand-ins for the simulation data the
paper uses). Times are CUDA-event times of the library calls with the batch already in device memory.

  python -m paper_2412_16544_gb300.sweeps --which all --out results.jsonl
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

import paper_2412_16544_gb300 as B


def reshapes(grid: int) -> dict:
    """Tensorisations of a grid^3 snapshot (grid a power of two): each spatial mode split in C order,
    so the data are not moved. For 64^3 these are the shapes of App. D.2 without their variable, time
    and batch modes (2^18 as (2, 2, 4)^4 x 2 x 2: 14 modes)."""
    k = int(round(np.log2(grid)))
    if 2 ** k != grid:
        raise ValueError("grid must be a power of two")
    out = {f"{grid}^3": (grid,) * 3}
    if k % 2 == 0:
        out[f"{2 ** (k // 2)}^6"] = (2 ** (k // 2),) * 6
        out[f"4^{3 * k // 2}"] = (4,) * (3 * k // 2)
    if grid == 64:
        out["(2x2x4)^4x2x2"] = (2, 2, 4) * 4 + (2, 2)
    return {n: s for n, s in out.items() if len(s) <= 16}


# permutations of the 8^6 item (x_hi, x_lo, y_hi, y_lo, z_hi, z_lo)
AXIS_ORDERS = {
    "baseline": (0, 1, 2, 3, 4, 5),
    "swap_xlo_zhi": (0, 4, 2, 3, 1, 5),
    "coarse_first": (0, 2, 4, 1, 3, 5),
    "reversed": (5, 4, 3, 2, 1, 0),
}


def _timed(fn):
    """(result, milliseconds) of a library call, with CUDA events on the current stream."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def _median_of(fn, repeats: int):
    """Run fn (which returns (state, ms)) `repeats` times after one untimed warm-up run; the median time.
    Every run but the last releases its state."""
    runs = []
    for i in range(repeats + 1):
        state, ms = fn()
        if i < repeats:
            B.bht_state_destroy(state)
        if i > 0:
            runs.append(ms)
    return state, float(np.median(runs))


def _status(fn):
    """Run fn; a capacity error of the library becomes a recorded failure (like an out-of-memory run)."""
    try:
        return fn(), None
    except B.BHTError as e:
        return None, str(e)


def reduction_ratio(state) -> float:
    r = B.bht_get_ranks(state)
    return float(np.prod(B.bht_get_dims(state))) / (r[1] * r[2])


def spectral_batch(seed: int, first: int, count: int, grid: int):
    import torch
    import bht_synth
    return torch.from_numpy(bht_synth.spectral_field(seed, first, count, n=grid)).cuda()


def bht_vs_ht(grid=64, batches=(8, 16, 32, 64, 128), eps_list=(0.1, 0.05),
              norms=("none", "maxabs", "unitvec", "zscore"), precision="mixed", seed=0, repeats=3):
    rows = []
    for N in batches:
        raw = spectral_batch(seed, 0, N, grid)
        for norm in norms:
            Y = raw.clone()
            B.bht_normalize(Y, norm)
            numel = Y.numel()
            for eps in eps_list:
                row = {"study": "bht_vs_ht", "grid": grid, "N": N, "eps": eps, "norm": norm, "precision": precision}
                tree = B.bht_tree_create_balanced(Y.shape[1:])
                (st, err) = _status(lambda: _median_of(lambda: _timed(lambda: B.bht_l2r(tree, Y, eps, precision=precision)),
                                                      repeats))
                if st is not None:
                    state, ms = st
                    row.update(bht_ms=ms, bht_cr=numel / B.bht_num_elements(state), bht_ranks=B.bht_get_ranks(state))
                    B.bht_state_destroy(state)
                else:
                    row["bht_failed"] = err
                B.bht_tree_destroy(tree)
                (st, err) = _status(lambda: _median_of(lambda: _timed(lambda: B.ht_l2r(Y, eps, precision=precision)), repeats))
                if st is not None:
                    state, ms = st
                    row.update(ht_ms=ms, ht_cr=numel / B.bht_num_elements(state), ht_ranks=B.bht_get_ranks(state))
                    B.bht_state_destroy(state)
                else:
                    row["ht_failed"] = err
                rows.append(row)
    return rows


def _stream(items, shape, eps, precision, inc, test, groups_per_item=1, norm="none", repeats=3):
    """BHT-l2r on the first increment, HT-RISE on the rest; items [M, ...] on the device, reshaped to
    `shape` per item. Returns time (median of `repeats` runs after a warm-up), CR, RR, RTE on the
    held-out items `test` (same shape and norm)."""
    M = items.shape[0]
    Y = items.reshape((M,) + tuple(shape))
    if norm != "none":
        B.bht_normalize(Y, norm, groups=M * groups_per_item)
        B.bht_normalize(test, norm, groups=test.shape[0] * groups_per_item)
    tree = B.bht_tree_create_balanced(shape)
    incs = [Y[k:k + inc].contiguous() for k in range(0, M, inc)]
    skipped = 0

    def one_run():
        nonlocal skipped
        skipped = 0
        st, total = _timed(lambda: B.bht_l2r(tree, incs[0], eps, precision=precision))
        for Yk in incs[1:]:
            info, ms = _timed(lambda: B.htrise_update(st, Yk, eps, precision=precision))
            total += ms
            skipped += int(info.skipped)
        return st, total

    st, total_ms = _median_of(one_run, repeats)
    rte = B.relative_test_error(st, test.reshape((test.shape[0],) + tuple(shape)).contiguous())
    out = {"ms": total_ms, "cr": Y.numel() / B.bht_num_elements(st), "rr": reduction_ratio(st), "rte": rte,
           "ranks": B.bht_get_ranks(st), "skipped_updates": skipped}
    B.bht_state_destroy(st)
    B.bht_tree_destroy(tree)
    return out


def reshape(grid=64, items=128, inc=16, test=16, eps=0.1, precision="mixed", seed=0):
    rows = []
    base = spectral_batch(seed, 0, items, grid)
    held = spectral_batch(seed, 10_000, test, grid)
    for name, shape in reshapes(grid).items():
        row = {"study": "reshape", "shape": name, "eps": eps, "items": items, "increment": inc, "precision": precision}
        res, err = _status(lambda: _stream(base, shape, eps, precision, inc, held.clone()))
        row.update(res if res is not None else {"failed": err})
        rows.append(row)
    return rows


def axis_order(items=128, inc=16, test=16, eps=0.1, precision="mixed", seed=0):
    rows = []
    base = spectral_batch(seed, 0, items, 64).reshape((items,) + (8,) * 6)
    held = spectral_batch(seed, 10_000, test, 64).reshape((test,) + (8,) * 6)
    for name, perm in AXIS_ORDERS.items():
        Yp = B.bht_permute_items(base.contiguous(), perm)
        Tp = B.bht_permute_items(held.contiguous(), perm)
        row = {"study": "axis_order", "order": name, "perm": list(perm), "eps": eps, "items": items,
               "increment": inc, "precision": precision}
        res, err = _status(lambda: _stream(Yp, Yp.shape[1:], eps, precision, inc, Tp))
        row.update(res if res is not None else {"failed": err})
        rows.append(row)
    return rows


def normalize(grid=48, items=64, inc=16, test=8, eps=1e-2, precision="mixed", seed=0, nvar=5):
    import torch
    import bht_synth
    rows = []
    base = torch.from_numpy(bht_synth.multivar_field(seed, 0, items, n=grid, nvar=nvar)).cuda()
    held = torch.from_numpy(bht_synth.multivar_field(seed, 10_000, test, n=grid, nvar=nvar)).cuda()
    for norm in ("none", "maxabs", "unitvec", "zscore"):
        row = {"study": "normalize", "norm": norm, "eps": eps, "items": items, "increment": inc, "precision": precision}
        res, err = _status(lambda: _stream(base.clone(), base.shape[1:], eps, precision, inc, held.clone(),
                                           groups_per_item=nvar, norm=norm))
        row.update(res if res is not None else {"failed": err})
        rows.append(row)
    return rows


def budget(grid=64, items=128, inc=32, test=16, eps_list=(1e-2, 1e-1), precision="mixed", seed=0):
    """Uniform node-wise tolerance (Algorithms 1, 2) against the adaptive budget of App. C on the same
    stream: CR, RR, RTE, time and the error actually spent per increment."""
    import torch
    rows = []
    base = spectral_batch(seed, 0, items, grid)
    held = spectral_batch(seed, 10_000, test, grid)
    for eps in eps_list:
        for mode in ("uniform", "adaptive"):
            tree = B.bht_tree_create_balanced(base.shape[1:])
            incs = [base[k:k + inc].contiguous() for k in range(0, items, inc)]

            def one_run():
                st, total = _timed(lambda: B.bht_l2r(tree, incs[0], eps, precision=precision, budget=mode))
                for Yk in incs[1:]:
                    _, ms = _timed(lambda: B.htrise_update(st, Yk, eps, precision=precision))
                    total += ms
                return st, total

            st, ms = _median_of(one_run, 3)
            errs = []
            for k, Yk in enumerate(incs):
                rec = B.ht_reconstruct(st, k * inc, Yk.shape[0], dtype="float32")
                errs.append(float(torch.linalg.vector_norm(rec - Yk) / torch.linalg.vector_norm(Yk)))
            rows.append({"study": "budget", "budget": mode, "eps": eps, "items": items, "increment": inc,
                         "precision": precision, "ms": ms, "cr": base.numel() / B.bht_num_elements(st),
                         "rr": reduction_ratio(st), "rte": B.relative_test_error(st, held),
                         "max_err_over_eps": max(errs) / eps, "ranks": B.bht_get_ranks(st)})
            B.bht_state_destroy(st)
            B.bht_tree_destroy(tree)
    return rows


STUDIES = {"bht_vs_ht": bht_vs_ht, "reshape": reshape, "axis_order": axis_order, "normalize": normalize,
           "budget": budget}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="all", help="comma-separated: " + ",".join(STUDIES) + " or all")
    ap.add_argument("--out", default=None, help="append JSON lines here as well as to stdout")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--small", action="store_true", help="reduced sizes (a quick check)")
    a = ap.parse_args()
    names = list(STUDIES) if a.which == "all" else a.which.split(",")
    small = {
        "bht_vs_ht": dict(grid=32, batches=(8, 16), eps_list=(0.1,), norms=("none", "zscore")),
        "reshape": dict(grid=16, items=16, inc=8, test=4),
        "axis_order": dict(items=16, inc=8, test=4),
        "normalize": dict(grid=16, items=16, inc=8, test=4),
        "budget": dict(grid=16, items=16, inc=8, test=4, eps_list=(1e-1,)),
    }
    t0 = time.time()
    for name in names:
        kw = dict(small[name]) if a.small else {}
        for row in STUDIES[name](precision=a.precision, **kw):
            line = json.dumps(row)
            print(line, flush=True)
            if a.out:
                with open(a.out, "a") as f:
                    f.write(line + "\n")
    print(json.dumps({"seconds": time.time() - t0}))


if __name__ == "__main__":
    main()

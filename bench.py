#!/usr/bin/env python
"""Throughput of the batch hierarchical Tucker hot path (BHT-l2r + HT-RISE) on GB300.

One step = one pass of the whole path over one synthetic stream: BHT-l2r
(Algorithm 1) on the first increment, HT-RISE (Algorithm 2) on each later
increment. Default workload: the 64^3 advected spectral field, 20 increments of
32 snapshots (671 MB of fp32), eps_rel = 1e-2, inputs resident in HBM when the
timed region starts. The metric is GB/s of fp32 stream compressed.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of tensor stream compressed (BHT-l2r+HT-RISE) at rel err<=eps, fast vs plain FP64"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default=os.environ.get("BHT_BENCH_PRECISION", "mixed"))
    ap.add_argument("--eps", type=float, default=None, help="default: 1e-2 (spectral, sensor), 1e-3 (bumps, multivar)")
    ap.add_argument("--increments", type=int, default=None, help="default: 20 (spectral), 4 (bumps, sensor, multivar)")
    ap.add_argument("--items", type=int, default=None, help="default: 32 (spectral), 8 (bumps), 64 (sensor)")
    ap.add_argument("--grid", type=int, default=64, help="edge of the cubic snapshot")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", choices=["spectral", "bumps", "sensor", "multivar"], default="spectral",
                    help="spectral: the 64^3 advected field stream (the headline); bumps: 16^3 Gaussian bumps, FP64 "
                         "items; sensor: 24^5 Chebyshev sensor responses; multivar: 16 independent streams of "
                         "5 x 48^3 items with increment sizes U{1..64}, compressed concurrently")
    ap.add_argument("--streams", type=int, default=16)
    a = ap.parse_args(argv)
    defaults = {"spectral": (1e-2, 20, 32), "bumps": (1e-3, 4, 8), "sensor": (1e-2, 4, 64), "multivar": (1e-3, 4, 0)}
    eps, inc, items = defaults[a.workload]
    a.eps = eps if a.eps is None else a.eps
    a.increments = inc if a.increments is None else a.increments
    a.items = items if a.items is None else a.items
    return a


def item_dims(a):
    return {"spectral": (a.grid,) * 3, "bumps": (16, 16, 16), "sensor": (24,) * 5}[a.workload]


def workload_name(a):
    what = {"spectral": f"advected spectral field {a.grid}^3 (|k|<=16, |k|^-5/3)",
            "bumps": "16^3 Gaussian bumps (5 separable terms, FP64 items)",
            "sensor": "24^5 Chebyshev sensor responses (20 separable degree-6 terms + 0.01 N(0,1))"}[a.workload]
    return f"{what}, {a.increments} increments x {a.items} items, eps_rel={a.eps:g}"


def gen_stream(a, seed):
    import bht_synth
    n = a.increments * a.items
    if a.workload == "bumps":
        Y = bht_synth.gaussian_bumps(seed, 0, n)
    elif a.workload == "sensor":
        Y = bht_synth.chebyshev_sensor(seed, 0, n)
    else:
        Y = bht_synth.spectral_field(seed, 0, n, n=a.grid)
    return Y.reshape((a.increments, a.items) + item_dims(a))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the reference arm: the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(Yhost, eps, seconds):
    """BHT-l2r on increment 1, then HT-RISE while the budget lasts. Returns (bytes, s, increments, state)."""
    import oracle
    t0 = time.perf_counter()
    st = oracle.bht_l2r(Yhost[0], eps)
    done = 1
    while done < len(Yhost) and time.perf_counter() - t0 < seconds:
        oracle.htrise_update(st, Yhost[done], eps)
        done += 1
    dt = time.perf_counter() - t0
    return done * Yhost[0].nbytes, dt, done, st


def run_reference(a, rank):
    if rank != 0:
        return
    Y = gen_stream(a, 0)
    nthreads = os.cpu_count()
    for _ in range(a.warmup):
        oracle_sample(Y, a.eps, 1.0)  # BHT-l2r on increment 1 at least
    times, nbytes, incs = [], 0, 0
    for _ in range(a.steps):
        b, dt, done, _ = oracle_sample(Y, a.eps, min(a.cpu_seconds, 8.0))
        times.append(dt)
        nbytes, incs = b, done
    ms = 1000.0 * statistics.mean(times)
    gbs = nbytes / (ms / 1000.0) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "sample": f"first {incs} of {a.increments} increments per step"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"BHT-l2r on increment 1 + HT-RISE on increments 2..{incs} (numpy FP64)"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# kernel source identity (for the DRAM traffic recorded from ncu)
# ---------------------------------------------------------------------------
# class -> (file, the device functions whose text does the class's work, headers of device helpers they use)
KERNEL_SOURCES = {
    "eig_tridiag_f64": ("paper_2412_16544_gb300/csrc/eig.cu", ["tridiag_rows_kernel", "householder"],
                        ["paper_2412_16544_gb300/csrc/sync.cuh"]),
}


def function_text(src: str, name: str) -> str:
    """The text of the device function `name` in `src`: from its declaration line to its matching brace."""
    m = re.search(r"^[^\n;{}]*__(?:global|device)__[^\n;{}]*\b" + re.escape(name) + r"\(", src, flags=re.M)
    if not m:
        raise KeyError(name)
    i = src.index("{", m.end())
    depth = 0
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[m.start():j + 1]
    raise ValueError(name)


def kernel_source_hash(cls: str):
    """sha256 of the source text a kernel class's work depends on, or None when it cannot be read."""
    if cls not in KERNEL_SOURCES:
        return None
    path, funcs, headers = KERNEL_SOURCES[cls]
    try:
        src = open(os.path.join(ROOT, path)).read()
        parts = [function_text(src, fn) for fn in funcs] + [open(os.path.join(ROOT, h)).read() for h in headers]
    except (OSError, KeyError, ValueError):
        return None
    return hashlib.sha256("\n".join(parts).encode()).hexdigest()


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
# algorithmic work per kernel class is attached by the library to every launch
PEAK_FP64_TFLOPS = 1.25  # FP64 nominal of the profiling recipe table (no measured FP64 peak is provided)


def run_ours(a, rank, world, local_rank):
    import torch
    import paper_2412_16544_gb300 as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    Yh = gen_stream(a, seed=rank)                  # each rank compresses its own independent stream
    Yd = torch.from_numpy(Yh).to(dev)              # resident in HBM before the timed region
    bytes_per_step = Yh.nbytes
    tree = B.bht_tree_create_balanced(list(item_dims(a)))
    stream = torch.cuda.current_stream()

    def one_pass(prec, src):
        st = B.bht_l2r(tree, src[0], a.eps, precision=prec)
        skips = 0
        for k in range(1, a.increments):
            info = B.htrise_update(st, src[k], a.eps, precision=prec)
            skips += int(info.skipped)
        return st, skips

    L2_BYTES = 129 * 1024 * 1024
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if bytes_per_step <= L2_BYTES else None

    def timed(prec, steps, warmup, profile_mask=0):
        for _ in range(warmup):
            st, _ = one_pass(prec, Yd)
            B.bht_state_destroy(st)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        B.bht_launch_count(reset=True)
        B.bht_profile_read(reset=True)
        B.bht_profile_enable(profile_mask)
        sampler = ClockSampler(local_rank)
        sampler.start()
        time.sleep(0.3)
        states = []
        total_ms = 0.0
        for _ in range(steps):
            if flush is not None:
                flush.add_(1)  # a write larger than L2 between timed steps (small workloads only)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, skips = one_pass(prec, Yd)
            e1.record(stream)
            states.append((st, skips))
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
        clocks = sampler.stop()
        B.bht_profile_enable(0)
        launches = B.bht_launch_count(reset=True)
        prof = B.bht_profile_read(reset=True, work=True)
        ms = job_max(dist, total_ms / steps, dev)
        if dist is not None:
            dist.barrier()
        return ms, launches / steps, prof, clocks, states

    # profiled pass: which kernel class dominates (all classes timed)
    B.bht_profile_read(reset=True)
    B.bht_profile_enable((1 << B.KERNEL_CLASSES) - 1)
    st, _ = one_pass(a.precision, Yd)
    torch.cuda.synchronize()
    B.bht_profile_enable(0)
    breakdown = B.bht_profile_read(reset=True)
    B.bht_state_destroy(st)
    dom_name = max(breakdown, key=lambda k: breakdown[k][0])
    dom_cls = [B.bht_kernel_class_name(i) for i in range(B.KERNEL_CLASSES)].index(dom_name)
    hbm_peak = 6800.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak_src = "fallback 6.8 TB/s (profiling recipe)"
    if os.path.exists(peaks_path):
        hbm_peak = float(json.load(open(peaks_path)).get("hbm_gbs", hbm_peak))
        peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)"

    names = [B.bht_kernel_class_name(i) for i in range(B.KERNEL_CLASSES)]
    tc_cls = names.index("ttm_tc")
    ms, launches, prof, clocks, states = timed(a.precision, a.steps, a.warmup,
                                               profile_mask=(1 << dom_cls) | (1 << tc_cls))
    value = job_rate_gbs(bytes_per_step, world, ms / 1000.0)

    # accuracy of the last timed pass: per-increment relative error of the reconstruction
    st, skips = states[-1]
    ranks = B.bht_get_ranks(st)
    errs = []
    for k in sorted({0, 1, a.increments // 2, a.increments - 1}):
        rec = B.ht_reconstruct(st, k * a.items, a.items, dtype="float32")
        errs.append(float(torch.linalg.vector_norm(rec - Yd[k]) / torch.linalg.vector_norm(Yd[k])))
    cores = B.bht_num_elements(st)
    cr = Yh.size / cores
    for s_, _ in states:
        B.bht_state_destroy(s_)

    # the plain FP64 GPU arm, for the fast-vs-plain comparison
    plain = None
    if a.precision != "fp64" and not a.no_fp64_arm:
        ms64, _, _, _, st64 = timed("fp64", 1, 1)
        for s_, _ in st64:
            B.bht_state_destroy(s_)
        plain = {"value": job_rate_gbs(bytes_per_step, world, ms64 / 1000.0), "unit": "GB/s", "ms_per_step": ms64}

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not a.no_e2e:
        Yp = torch.from_numpy(Yh).pin_memory()
        # the result read back: the root of the whole accumulation, into pinned host memory
        st_w, _ = one_pass(a.precision, Yp)      # one untimed pass through the host path
        r = B.bht_get_ranks(st_w)
        root_host = torch.empty((a.increments * a.items, r[1], r[2]), dtype=torch.float64).pin_memory()
        B.bht_state_destroy(st_w)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        st_e, _ = one_pass(a.precision, Yp)
        rr = B.bht_get_ranks(st_e)
        if (rr[1], rr[2]) != (r[1], r[2]):  # ranks can differ only by run-to-run rounding at a tie
            root_host = torch.empty((a.increments * a.items, rr[1], rr[2]), dtype=torch.float64).pin_memory()
        root = B.bht_get_root(st_e, 0, a.increments * a.items, out=root_host)
        torch.cuda.synchronize()
        dt = job_max(dist, time.perf_counter() - t0, dev)
        e2e = {"value": job_rate_gbs(bytes_per_step, world, dt), "unit": "GB/s",
               "h2d_bytes_per_step": int(Yh.nbytes), "d2h_bytes_per_step": int(root.numel() * 8)}
        B.bht_state_destroy(st_e)

    # CPU baseline: the oracle on a bounded sample, rank 0 only
    cpu = None
    oracle_diff = None
    if rank == 0 and not a.no_cpu_baseline:
        nb, dt, incs, ost = oracle_sample(Yh, a.eps, a.cpu_seconds)
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"BHT-l2r on increment 1 + HT-RISE on increments 2..{incs} of the same stream "
                         f"({nb / 1e6:.0f} MB, numpy FP64)"}
        import oracle
        st1 = B.bht_l2r(tree, Yd[0], a.eps, precision=a.precision)
        r_gpu = B.ht_reconstruct(st1, 0, a.items, dtype="float64").cpu().numpy()
        r_or = oracle.reconstruct(ost, 0, a.items)
        oracle_diff = float(np.linalg.norm(r_gpu - r_or) / np.linalg.norm(Yh[0]))
        B.bht_state_destroy(st1)

    # roofline of the dominant kernel class and of the tensor-core mode product (algorithmic work per launch
    # accumulated by the library, CUDA-event durations on the launch stream over the timed region)
    def traffic_of(name):
        # per-launch DRAM bytes from a committed ncu capture, only while the kernel's source is unchanged
        path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
        try:
            lines = open(path).read().splitlines()
        except OSError:
            return None
        tag = f"spectral{a.grid}" if a.workload == "spectral" and a.eps == 1e-2 else None
        for ln in lines:
            f = ln.split()
            if len(f) == 5 and not ln.startswith("#") and f[0] == tag and f[1] == name:
                h = kernel_source_hash(name) if f[3] == "kernel-source" else None
                return float(f[2]) if h is not None and h == f[4] else None
        return None

    def roof(name):
        t_ms, n_l, flops, nbytes = prof.get(name, (0.0, 0, 0.0, 0.0))
        if not n_l or t_ms <= 0:
            return None
        per_launch_s = t_ms / n_l / 1000.0
        if name in ("ttm_tc", "copy", "norm"):
            ach = nbytes / n_l / per_launch_s / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                    "traffic": traffic_of(name), "kernel": name, "launches_per_step": n_l / a.steps,
                    "ms_per_launch": per_launch_s * 1e3, "peak_source": peak_src}
        if name.endswith("f32"):
            peak = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA lanes x 2 flops x max SM clock
            src = "FP32 SIMT: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz"
        else:
            peak = PEAK_FP64_TFLOPS
            src = "FP64 nominal of the profiling recipe (1.25 TFLOP/s)"
        ach = flops / n_l / per_launch_s / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic_of(name), "kernel": name, "launches_per_step": n_l / a.steps,
                "ms_per_launch": per_launch_s * 1e3, "peak_source": src}

    roofline = roof(dom_name)
    roofline_tc = roof("ttm_tc")

    if dist is not None:
        dist.barrier()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32" if a.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "precision": a.precision, "items_per_step": a.increments * a.items,
                   "bytes_per_step": bytes_per_step, "parallelism": f"{world} independent streams",
                   "l2": (f"inputs ({bytes_per_step / 1e6:.0f} MB per stream) larger than L2 (129 MB); no flush"
                          if flush is None else
                          f"inputs ({bytes_per_step / 1e6:.1f} MB) smaller than L2: a 258 MB write flushes L2 "
                          f"before every timed step (outside the timed region)")},
        "roofline": roofline, "roofline_ttm_tc": roofline_tc, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks,
        "plain_fp64": plain,
        "accuracy": {"max_rel_err_per_increment": max(errs), "eps_rel": a.eps,
                     "rel_diff_vs_oracle_increment1": oracle_diff},
        "stream": {"ranks": ranks, "skipped_updates": skips, "updates": a.increments - 1, "compression_ratio": cr},
        "kernel_breakdown_ms": {k: round(v[0], 4) for k, v in breakdown.items() if v[1]},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_multistream(a):
    """Independent streams compressed at once, one host thread and one CUDA stream each, against the same
    streams one after another; the 5 x 48^3 multi-variable fields, eps = 1e-3 unless given."""
    import threading
    import torch
    import bht_synth
    import paper_2412_16544_gb300 as B

    eps = a.eps
    incs = a.increments
    data, total = [], 0
    for sidx in range(a.streams):
        sizes = [int(x) for x in bht_synth.increment_sizes(sidx, incs)]
        Y = torch.from_numpy(bht_synth.multivar_field(sidx, 0, sum(sizes))).cuda()
        total += Y.numel() * 4
        data.append(list(torch.split(Y, sizes)))
    tree = B.bht_tree_create_balanced([5, 48, 48, 48])

    def one_stream(batches, cs, out, i):
        with torch.cuda.stream(cs):
            st = B.bht_l2r(tree, batches[0], eps, precision=a.precision, stream=cs)
            for Yk in batches[1:]:
                B.htrise_update(st, Yk, eps, precision=a.precision, stream=cs)
            out[i] = st

    def run(concurrent):
        states = [None] * a.streams
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if concurrent:
            cs = [torch.cuda.Stream() for _ in range(a.streams)]
            th = [threading.Thread(target=one_stream, args=(data[i], cs[i], states, i)) for i in range(a.streams)]
            for t in th:
                t.start()
            for t in th:
                t.join()
        else:
            cs = torch.cuda.current_stream()
            for i in range(a.streams):
                one_stream(data[i], cs, states, i)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if any(x is None for x in states):
            raise RuntimeError("a stream failed")
        return dt, states

    for _ in range(a.warmup):
        _, sts = run(True)
        for x in sts:
            B.bht_state_destroy(x)
    t_conc, t_seq = [], []
    for _ in range(a.steps):
        dt, sts = run(True)
        t_conc.append(dt)
        for x in sts:
            B.bht_state_destroy(x)
    dt, sts = run(False)
    t_seq.append(dt)
    errs = []
    for i, x in enumerate(sts):
        first = 0
        for Yk in data[i]:
            rec = B.ht_reconstruct(x, first, Yk.shape[0], dtype="float32")
            errs.append(float(torch.linalg.vector_norm(rec - Yk) / torch.linalg.vector_norm(Yk)))
            first += Yk.shape[0]
        B.bht_state_destroy(x)
    ms = 1000.0 * statistics.median(t_conc)
    line = {
        "metric": METRIC, "value": total / (ms / 1000.0) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32" if a.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": f"{a.streams} independent multi-variable streams 5x48^3, {incs} increments of "
                               f"U{{1..64}} items each, eps_rel={eps:g}", "precision": a.precision,
                   "bytes_per_step": total, "timing": "host wall clock around all streams, device synchronised"},
        "sequential": {"value": total / t_seq[0] / 1e9, "unit": "GB/s", "ms_per_step": 1000.0 * t_seq[0]},
        "accuracy": {"max_rel_err_per_increment": max(errs), "eps_rel": eps},
    }
    print(json.dumps(line), flush=True)
    B.bht_tree_destroy(tree)


def rank_env():
    """(rank, world size, local rank) from the torchrun environment; (0, 1, 0) when launched alone."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_max(dist, value, device="cpu"):
    """Maximum of a per-rank scalar over the job (the slowest rank sets the job's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate_gbs(bytes_per_rank, world, seconds_max):
    """Whole-job throughput: every rank compresses its own stream of bytes_per_rank in the job's time."""
    return bytes_per_rank * world / seconds_max / 1e9


def main():
    a = parse()
    rank, world, local_rank = rank_env()
    if a.impl == "reference":
        run_reference(a, rank)
        return
    if a.workload == "multivar":
        run_multistream(a)
        return
    run_ours(a, rank, world, local_rank)


if __name__ == "__main__":
    main()

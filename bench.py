#!/usr/bin/env python
"""Throughput of the batch hierarchical Tucker hot path (BHT-l2r + HT-RISE) on GB300.

One step = one pass of the whole path over one synthetic stream: BHT-l2r
(Algorithm 1) on the first increment, HT-RISE (Algorithm 2) on each later
increment. Default workload: the 24^5 Chebyshev sensor-grid stream, 50
increments of 64 items (2.04 GB of fp32 each, 102 GB in all), eps_rel = 1e-2,
drawn on the device before the timed region (the inputs are resident in HBM
when it starts). The metric is GB/s of fp32 stream compressed. The 64^3
advected spectral-field stream (20 x 32, eps_rel = 1e-2) is measured in the
same run as a second record.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of tensor stream compressed (BHT-l2r+HT-RISE) at rel err<=eps, fast vs plain FP64"
L2_BYTES = 129 * 1024 * 1024
FP64_LA = ("eig_tridiag_f64", "eig_bisect_f64", "gemm_f64", "eig_vec_f64", "eig_back_f64", "house_f64", "spd_test_f64", "ritz_small")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default=os.environ.get("BHT_BENCH_PRECISION", "mixed"))
    ap.add_argument("--eps", type=float, default=None, help="default: 1e-2 (sensor, spectral), 1e-3 (bumps, multivar)")
    ap.add_argument("--increments", type=int, default=None, help="default: 50 (sensor), 20 (spectral), 4 (bumps)")
    ap.add_argument("--items", type=int, default=None, help="default: 64 (sensor), 32 (spectral), 8 (bumps)")
    ap.add_argument("--grid", type=int, default=64, help="edge of the cubic snapshot (spectral)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true")
    ap.add_argument("--no-second", action="store_true", help="skip the 64^3 spectral-field second record")
    ap.add_argument("--roofline-steps", type=int, default=2)
    ap.add_argument("--per-batch", action="store_true",
                    help="one htrise_update call per increment instead of one htrise_update_stream call")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", choices=["sensor", "spectral", "bumps", "multivar"], default="sensor",
                    help="sensor: 24^5 Chebyshev sensor responses drawn on the device (the headline); spectral: the "
                         "64^3 advected field; bumps: 16^3 Gaussian bumps, FP64 items; multivar: 16 independent "
                         "streams of 5 x 48^3 items with increment sizes U{1..64}, compressed concurrently")
    ap.add_argument("--streams", type=int, default=16)
    a = ap.parse_args(argv)
    defaults = {"sensor": (1e-2, 50, 64), "spectral": (1e-2, 20, 32), "bumps": (1e-3, 4, 8), "multivar": (1e-3, 4, 0)}
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


# ---------------------------------------------------------------------------
# streams
# ---------------------------------------------------------------------------
class Stream:
    """The increments of one stream on the device, and host copies of parts of it on demand."""

    def __init__(self, a, seed, dev):
        import torch
        import bht_synth
        import paper_2412_16544_gb300 as B
        self.a, self.seed = a, seed
        shape = (a.increments, a.items) + item_dims(a)
        if a.workload == "sensor":
            # coefficients on the host (numpy, per item), the items on the device (bht_synth_chebyshev)
            c = bht_synth.chebyshev_coefficients(seed, 0, a.increments * a.items)
            self.Y = torch.empty(shape, dtype=torch.float32, device=dev)
            for k in range(a.increments):
                B.bht_synth_chebyshev(c[k * a.items:(k + 1) * a.items], 24, seed=seed, first_item=k * a.items,
                                      out=self.Y[k])
            torch.cuda.synchronize(dev)
            self.where = "drawn on the device (bht_synth_chebyshev), coefficients and noise counters as bht_synth"
        else:
            Yh = gen_stream(a, seed)
            self.Y = torch.from_numpy(Yh).to(dev)
            self.where = "drawn on the host (bht_synth), copied to the device once"
        self.inc = [self.Y[k] for k in range(a.increments)]
        self.nbytes = self.Y.numel() * self.Y.element_size()

    def host_items(self, k, first, count):
        """Items first .. first+count-1 of increment k as a float64 numpy array (the data the GPU compressed)."""
        return self.Y[k, first:first + count].double().cpu().numpy()


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


def oracle_chunks(a, stream_or_host):
    """The oracle's bounded sample: the stream's increments, or for the 24^5 stream chunks of 4 items of
    increment 1 (a whole increment is about a minute of host time per call)."""
    if a.workload == "sensor":
        chunk = 4
        if isinstance(stream_or_host, Stream):
            return [stream_or_host.host_items(0, chunk * j, chunk) for j in range(a.items // chunk)], chunk
        import bht_synth
        return [bht_synth.chebyshev_sensor(0, chunk * j, chunk).astype(np.float64) for j in range(4)], chunk
    return [x for x in stream_or_host], a.items


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.rows = []

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
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                self.rows.append((ts, float(f[2]), float(f[3]), f[6], f[7], f[8], f[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in self.rows), "sm_max_mhz": max(r[2] for r in self.rows),
                "reasons": reasons, "samples": len(self.rows)}

    def median_between(self, t0, t1):
        v = [r[1] for r in self.rows if t0 <= r[0] <= t1]
        return statistics.median(v) if v else None


# ---------------------------------------------------------------------------
# the reference arm: the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(chunks, eps, seconds):
    """BHT-l2r on the first chunk, then HT-RISE on the next ones while the budget lasts.
    Returns (bytes of fp32 input compressed, seconds, chunks done, state)."""
    import oracle
    t0 = time.perf_counter()
    st = oracle.bht_l2r(chunks[0], eps)
    done = 1
    while done < len(chunks) and time.perf_counter() - t0 < seconds:
        oracle.htrise_update(st, chunks[done], eps)
        done += 1
    dt = time.perf_counter() - t0
    return sum(c.size * 4 for c in chunks[:done]), dt, done, st


def run_reference(a, rank):
    if rank != 0:
        return
    if a.workload == "sensor":
        chunks, per = oracle_chunks(a, None)
        budget = 0.0   # BHT-l2r on the first 4 items only: about 5 s per step on 16 cores
        sample = "BHT-l2r on items 0..3 of increment 1 (numpy FP64); a whole increment takes about a minute"
    else:
        chunks, per = oracle_chunks(a, gen_stream(a, 0))
        budget = min(a.cpu_seconds, 8.0)
        sample = None
    nthreads = os.cpu_count()
    for _ in range(a.warmup):
        oracle_sample(chunks, a.eps, 0.0)
    times, nbytes, done = [], 0, 0
    for _ in range(a.steps):
        b, dt, done, _ = oracle_sample(chunks, a.eps, budget)
        times.append(dt)
        nbytes = b
    ms = 1000.0 * statistics.mean(times)
    gbs = nbytes / (ms / 1000.0) / 1e9
    if sample is None:
        sample = f"BHT-l2r on increment 1 + HT-RISE on increments 2..{done} (numpy FP64)"
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "precision": a.precision,
                   "sample": f"{done} chunk(s) of {per} items per step"},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": nthreads, "kind": "oracle", "sample": sample},
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
    "pair_proj": ("paper_2412_16544_gb300/csrc/pair.cu", ["pair_project_ws_kernel", "ds_add", "ffma2"],
                  ["paper_2412_16544_gb300/csrc/tma.cuh"]),
    "pair_gram": ("paper_2412_16544_gb300/csrc/pair.cu", ["pair_gram24_kernel", "g24_block", "g24_fold"],
                  ["paper_2412_16544_gb300/csrc/tma.cuh"]),
}


def function_text(src: str, name: str) -> str:
    """The text of the device function `name` in `src`: from its declaration line to its matching brace."""
    m = re.search(r"^[^\n;{}]*__(?:global|device)__[^;{}]*?\b" + re.escape(name) + r"\(", src, flags=re.M)
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


def traffic_of(tag, name):
    """Per-launch DRAM bytes from a committed ncu capture, only while the kernel's source is unchanged."""
    try:
        lines = open(os.path.join(ROOT, "profiles", "dram_traffic.txt")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = ln.split()
        if len(f) == 5 and not ln.startswith("#") and f[0] == tag and f[1] == name:
            h = kernel_source_hash(name) if f[3] == "kernel-source" else None
            return float(f[2]) if h is not None and h == f[4] else None
    return None


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def measured_peaks(B):
    """(HBM GB/s and its source, FP64 TFLOP/s, FP32 TFLOP/s) for the rooflines."""
    hbm, src = 6800.0, "fallback 6.8 TB/s (profiling recipe)"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        hbm = float(json.load(open(path)).get("hbm_gbs", hbm))
        src = "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    f64 = max(B.bht_probe_fma_rate("float64") for _ in range(2))
    f32 = max(B.bht_probe_fma_rate("float32") for _ in range(2))
    return hbm, src, f64, f32


PER_BATCH = False  # --per-batch: one htrise_update call per increment instead of htrise_update_stream


def consecutive(incs):
    """incs[1:] as one [count][items]... view when they lie back to back in memory, else None."""
    import torch
    rest = incs[1:]
    if not rest or not all(isinstance(x, torch.Tensor) and x.is_contiguous() for x in rest):
        return None
    first = rest[0]
    for k, x in enumerate(rest):
        if x.shape != first.shape or x.data_ptr() != first.data_ptr() + k * first.numel() * first.element_size():
            return None
    return torch.as_strided(first, (len(rest),) + tuple(first.shape), (first.numel(),) + tuple(first.stride()))


def one_pass(B, tree, incs, eps, prec, infos=None):
    """BHT-l2r on the first increment, HT-RISE on the rest: one htrise_update_stream call over the rest
    (the library overlaps each increment's projection with the previous one's skip test), or one
    htrise_update call per increment."""
    st = B.bht_l2r(tree, incs[0], eps, precision=prec)
    rest = None if PER_BATCH else consecutive(incs)
    if rest is not None:
        got = B.htrise_update_stream(st, rest, eps, precision=prec)
    else:
        got = [B.htrise_update(st, incs[k], eps, precision=prec) for k in range(1, len(incs))]
    if infos is not None:
        infos.extend(got)
    return st, sum(int(i.skipped) for i in got)


def run_timed(B, torch, tree, incs, eps, prec, steps, warmup, dist, dev, local_rank, profile_mask=0, flush=None,
              clocks=True):
    """Warm-up passes, then `steps` passes timed with CUDA events on the launch stream, max over ranks."""
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        st, _ = one_pass(B, tree, incs, eps, prec)
        B.bht_state_destroy(st)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    B.bht_launch_count(reset=True)
    B.bht_batch_reads(reset=True)
    B.bht_profile_read(reset=True)
    B.bht_profile_enable(profile_mask)
    sampler = ClockSampler(local_rank) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    per_step, windows, states = [], [], []
    for _ in range(steps):
        if flush is not None:
            flush.add_(1)  # a write larger than L2 between timed steps (small workloads only)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        t0 = time.time()
        e0.record(stream)
        st, skips = one_pass(B, tree, incs, eps, prec, infos)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        windows.append((t0, time.time()))
        per_step.append(e0.elapsed_time(e1))
        states.append((st, skips, infos))
    clk = sampler.stop() if sampler else None
    B.bht_profile_enable(0)
    launches = B.bht_launch_count(reset=True)
    reads = B.bht_batch_reads(reset=True)
    prof = B.bht_profile_read(reset=True, work=True)
    ms = job_max(dist, sum(per_step) / steps, dev)
    if dist is not None:
        dist.barrier()
    by_clock = None
    if sampler and clk.get("samples"):
        bins = {}
        for (w0, w1), t in zip(windows, per_step):
            f = sampler.median_between(w0, w1)
            key = None if f is None else int(round(f / 15.0) * 15)
            bins.setdefault(key, []).append(t)
        by_clock = [{"sm_mhz": k, "steps": len(v), "ms_per_step": statistics.mean(v)} for k, v in sorted(
            bins.items(), key=lambda x: (x[0] is None, x[0]))]
    return {"ms": ms, "per_step": per_step, "launches": launches / steps, "reads": reads / steps, "prof": prof,
            "clocks": clk, "by_clock": by_clock, "states": states}


def accuracy(B, torch, st, incs, eps, items):
    """max over sampled increments of ||Y_k - Y~_k|| / ||Y_k||."""
    errs = []
    n = len(incs)
    for k in sorted({0, 1, n // 2, n - 1} & set(range(n))):
        rec = B.ht_reconstruct(st, k * items, items, dtype="float32")
        errs.append(float(torch.linalg.vector_norm((rec - incs[k]).double()) /
                          torch.linalg.vector_norm(incs[k].double())))
        del rec
    return max(errs)


def roofline_of(name, prof, steps, hbm, hbm_src, f64, f32, tag):
    """Roofline of one kernel class from the library's per-launch CUDA events: bound by HBM when its
    algorithmic intensity is below the ridge of the unit it computes on, else by that unit."""
    t_ms, n_l, flops, nbytes = prof.get(name, (0.0, 0, 0.0, 0.0))
    if not n_l or t_ms <= 0:
        return None
    per_launch_s = t_ms / n_l / 1000.0
    if name.endswith("f64"):
        peak_f, unit_src = f64, f"FP64 FMA probe of this run ({f64:.3f} TFLOP/s)"
    elif name == "ttm_tc":
        peak_f, unit_src = 0.0, "tensor pipe (not the bound)"
    else:
        peak_f, unit_src = f32, f"FP32 FMA probe of this run ({f32:.1f} TFLOP/s)"
    ai = flops / nbytes if nbytes > 0 else float("inf")
    ridge = peak_f * 1e12 / (hbm * 1e9) if peak_f > 0 else 0.0
    base = {"kernel": name, "launches_per_step": n_l / steps, "ms_per_launch": per_launch_s * 1e3,
            "traffic": traffic_of(tag, name), "timing": "CUDA events around every launch of the class on its stream, "
            "over separate timed steps (the headline steps run with the profiler off)"}
    if nbytes > 0 and (peak_f == 0.0 or ai < ridge):
        ach = nbytes / n_l / per_launch_s / 1e9
        return dict(base, bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                    peak_source=hbm_src + ", of measured")
    ach = flops / n_l / per_launch_s / 1e12
    return dict(base, bound="alu", achieved=ach, peak=peak_f, unit="TFLOP/s", frac=ach / peak_f,
                peak_source=unit_src + ", of measured")


def run_ours(a, rank, world, local_rank):
    import torch
    import paper_2412_16544_gb300 as B

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    hbm, hbm_src, f64, f32 = measured_peaks(B)
    S = Stream(a, seed=rank, dev=dev)            # each rank compresses its own independent stream
    tree = B.bht_tree_create_balanced(list(item_dims(a)))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if S.nbytes <= L2_BYTES else None
    tag = {"sensor": "sensor24", "spectral": f"spectral{a.grid}"}.get(a.workload, a.workload)

    # a profiled pass: every kernel class timed (which class dominates, FP64 linear-algebra share)
    B.bht_profile_read(reset=True)
    B.bht_profile_enable((1 << B.KERNEL_CLASSES) - 1)
    st, _ = one_pass(B, tree, S.inc, a.eps, a.precision)
    torch.cuda.synchronize(dev)
    B.bht_profile_enable(0)
    breakdown = B.bht_profile_read(reset=True)
    B.bht_state_destroy(st)
    names = [B.bht_kernel_class_name(i) for i in range(B.KERNEL_CLASSES)]
    dom_name = max(breakdown, key=lambda k: breakdown[k][0])
    total_ms = sum(v[0] for v in breakdown.values())
    la_share = sum(breakdown.get(k, (0.0, 0))[0] for k in FP64_LA) / total_ms if total_ms > 0 else None

    # the headline: the profiler off
    T = run_timed(B, torch, tree, S.inc, a.eps, a.precision, a.steps, a.warmup, dist, dev, local_rank, 0, flush)
    value = job_rate_gbs(S.nbytes, world, T["ms"] / 1000.0)
    st, skips, infos = T["states"][-1]
    ranks = B.bht_get_ranks(st)
    max_err = accuracy(B, torch, st, S.inc, a.eps, a.items)
    cores = B.bht_num_elements(st)
    cr = S.Y.numel() / cores
    upd_reads = [i.batch_reads for i in infos]
    skip_reads = [i.batch_reads for i in infos if i.skipped]
    exp_reads = [i.batch_reads for i in infos if not i.skipped]
    passes = {"per_increment": T["reads"] / a.increments,
              "bht_l2r": T["reads"] - sum(upd_reads),
              "skipped_update": statistics.mean(skip_reads) if skip_reads else None,
              "expanding_update": statistics.mean(exp_reads) if exp_reads else None,
              "counted": "kernels that read the whole input batch (bht_batch_reads)"}
    for s_, _, _ in T["states"]:
        B.bht_state_destroy(s_)

    # rooflines: the dominant class and the full-data passes, timed by the library's per-launch events
    # over separate steps
    cls = [dom_name] + [c for c in ("pair_proj", "pair_gram", "ttm_tc") if c != dom_name]
    mask = 0
    for c in cls:
        mask |= 1 << names.index(c)
    R = run_timed(B, torch, tree, S.inc, a.eps, a.precision, a.roofline_steps, 1, dist, dev, local_rank, mask, flush,
                  clocks=False)
    for s_, _, _ in R["states"]:
        B.bht_state_destroy(s_)
    roofline = roofline_of(dom_name, R["prof"], a.roofline_steps, hbm, hbm_src, f64, f32, tag)
    passes_roof = {c: roofline_of(c, R["prof"], a.roofline_steps, hbm, hbm_src, f64, f32, tag) for c in cls[1:]}

    # the plain FP64 GPU arm, for the fast-vs-plain comparison at equal reconstruction error
    plain = None
    if a.precision != "fp64" and not a.no_fp64_arm:
        # warmed on the first two increments only: a full FP64 pass of the 24^5 stream takes seconds
        st_w, _ = one_pass(B, tree, S.inc[:2], a.eps, "fp64")
        B.bht_state_destroy(st_w)
        P = run_timed(B, torch, tree, S.inc, a.eps, "fp64", 1, 0, dist, dev, local_rank, 0, flush, clocks=False)
        st64, _, _ = P["states"][-1]
        plain = {"value": job_rate_gbs(S.nbytes, world, P["ms"] / 1000.0), "unit": "GB/s", "ms_per_step": P["ms"],
                 "max_rel_err_per_increment": accuracy(B, torch, st64, S.inc, a.eps, a.items),
                 "ranks": B.bht_get_ranks(st64), "passes_per_increment": P["reads"] / a.increments}
        for s_, _, _ in P["states"]:
            B.bht_state_destroy(s_)

    # end to end through the public API with host (pinned) buffers
    e2e = None
    if not a.no_e2e:
        e2e = run_e2e(B, torch, tree, S, a, dist, dev, world)

    # CPU baseline: the oracle on a bounded sample, rank 0 only; both GPU arms against it on that sample
    cpu, oracle_diff = None, None
    if rank == 0 and not a.no_cpu_baseline:
        chunks, per = oracle_chunks(a, S if a.workload == "sensor" else [S.host_items(k, 0, a.items)
                                                                          for k in range(a.increments)])
        nb, dt, done, ost = oracle_sample(chunks, a.eps, a.cpu_seconds)
        what = (f"BHT-l2r on items 0..{per - 1} of increment 1 + HT-RISE on {done - 1} more chunk(s) of {per} items"
                if a.workload == "sensor" else f"BHT-l2r on increment 1 + HT-RISE on increments 2..{done}")
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": what + f" ({nb / 1e6:.0f} MB of fp32 input, numpy FP64); a rate on this sample, "
                                "extrapolated to the stream"}
        import oracle
        oracle_diff = {}
        for prec in ([a.precision, "fp64"] if a.precision != "fp64" else ["fp64"]):
            sub = [torch.from_numpy(np.ascontiguousarray(c)).to(dev).float() for c in chunks[:done]]
            stg, _ = one_pass(B, tree, sub, a.eps, prec)
            n_items = sum(c.shape[0] for c in chunks[:done])
            rg = B.ht_reconstruct(stg, 0, n_items, dtype="float64").cpu().numpy()
            ro = oracle.reconstruct(ost, 0, n_items)
            allc = np.concatenate(chunks[:done])
            oracle_diff[prec] = float(np.linalg.norm(rg - ro) / np.linalg.norm(allc))
            B.bht_state_destroy(stg)

    second = None
    if rank == 0 and not a.no_second and a.workload == "sensor" and world == 1:
        second = run_second(B, torch, dev, local_rank, a)

    if dist is not None:
        dist.barrier()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": T["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if a.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "precision": a.precision, "items_per_step": a.increments * a.items,
                   "bytes_per_step": S.nbytes, "parallelism": f"{world} independent streams", "inputs": S.where,
                   "api": ("bht_l2r + one htrise_update call per increment" if PER_BATCH else
                           "bht_l2r + one htrise_update_stream call over the other increments"),
                   "l2": (f"inputs ({S.nbytes / 1e9:.1f} GB per stream) larger than L2 (129 MB); no flush"
                          if flush is None else
                          f"inputs ({S.nbytes / 1e6:.1f} MB) smaller than L2: a 258 MB write flushes L2 "
                          f"before every timed step (outside the timed region)")},
        "roofline": roofline, "roofline_passes": passes_roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": T["launches"], "clocks": T["clocks"], "by_clock": T["by_clock"],
        "plain_fp64": plain,
        "accuracy": {"max_rel_err_per_increment": max_err, "eps_rel": a.eps,
                     "rel_diff_vs_oracle_on_sample": oracle_diff},
        "passes_over_y": passes,
        "fp64_la_share": la_share,
        "peaks": {"hbm_gbs": hbm, "fp64_tflops": f64, "fp32_tflops": f32,
                  "fp_source": "FMA probe of this run (bht_probe_fma_rate, CUDA events)"},
        "stream": {"ranks": ranks, "skipped_updates": skips, "updates": a.increments - 1, "compression_ratio": cr},
        "kernel_breakdown_ms": {k: round(v[0], 4) for k, v in breakdown.items() if v[1]},
        "second_record": second,
    }
    print(json.dumps(line), flush=True)
    B.bht_tree_destroy(tree)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(B, torch, tree, S, a, dist, dev, world):
    """One pass through the host path: every increment read from pinned host memory by the library's own
    staging copy, the root of the whole accumulation read back into pinned host memory."""
    try:
        Yp = torch.empty(S.Y.shape, dtype=S.Y.dtype, pin_memory=True)
    except RuntimeError:
        return {"value": None, "unit": "GB/s", "note": "pinned host memory for the whole stream unavailable"}
    for k in range(a.increments):
        Yp[k].copy_(S.Y[k])
    incs = [Yp[k] for k in range(a.increments)]
    st_w, _ = one_pass(B, tree, incs[:2], a.eps, a.precision)   # the host path warmed
    r_w = B.bht_get_ranks(st_w)
    B.bht_state_destroy(st_w)
    # the caller's pinned buffer for the root, like the inputs' before the timed region, sized from the
    # warm-up's ranks (the same stream); a rank that grows later gets a new buffer inside the timed region
    n_items = a.increments * a.items
    root_host = torch.empty((n_items, r_w[1], r_w[2]), dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    st_e, _ = one_pass(B, tree, incs, a.eps, a.precision)
    r = B.bht_get_ranks(st_e)
    if (r[1], r[2]) != (r_w[1], r_w[2]):
        root_host = torch.empty((n_items, r[1], r[2]), dtype=torch.float64, pin_memory=True)
    root = B.bht_get_root(st_e, 0, n_items, out=root_host)
    torch.cuda.synchronize(dev)
    dt = job_max(dist, time.perf_counter() - t0, dev)
    B.bht_state_destroy(st_e)
    out = {"value": job_rate_gbs(S.nbytes, world, dt), "unit": "GB/s", "h2d_bytes_per_step": int(S.nbytes),
           "d2h_bytes_per_step": int(root.numel() * 8),
           "note": "host wall clock; inputs and the root's pinned host buffer allocated before the timed region"}
    del Yp
    return out


def run_second(B, torch, dev, local_rank, a0):
    """The 64^3 advected spectral-field stream (20 x 32 snapshots, eps 1e-2): mixed and plain FP64 arms."""
    a = parse(["--workload", "spectral", "--steps", str(min(a0.steps, 5)), "--warmup", "2"])
    S = Stream(a, seed=0, dev=dev)
    tree = B.bht_tree_create_balanced(list(item_dims(a)))
    T = run_timed(B, torch, tree, S.inc, a.eps, "mixed", a.steps, a.warmup, None, dev, local_rank, 0, None)
    st, skips, _ = T["states"][-1]
    out = {"workload": workload_name(a), "value": S.nbytes / (T["ms"] / 1000.0) / 1e9, "unit": "GB/s",
           "ms_per_step": T["ms"], "steps": a.steps, "clocks": T["clocks"],
           "max_rel_err_per_increment": accuracy(B, torch, st, S.inc, a.eps, a.items),
           "ranks": B.bht_get_ranks(st), "skipped_updates": skips, "passes_per_increment": T["reads"] / a.increments}
    for s_, _, _ in T["states"]:
        B.bht_state_destroy(s_)
    P = run_timed(B, torch, tree, S.inc, a.eps, "fp64", 1, 1, None, dev, local_rank, 0, None, clocks=False)
    st64, _, _ = P["states"][-1]
    out["plain_fp64"] = {"value": S.nbytes / (P["ms"] / 1000.0) / 1e9, "unit": "GB/s", "ms_per_step": P["ms"],
                         "max_rel_err_per_increment": accuracy(B, torch, st64, S.inc, a.eps, a.items)}
    for s_, _, _ in P["states"]:
        B.bht_state_destroy(s_)
    B.bht_tree_destroy(tree)
    return out


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
        "dtype": "f32" if a.precision == "mixed" else "f64", "data": "synthetic",
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
    global PER_BATCH
    a = parse()
    PER_BATCH = a.per_batch
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

"""The multi-rank path of bench.py on CPU: world size 2 over gloo (127.0.0.1).

Each rank compresses its own stream (seed = rank), the job time is the maximum over ranks and the
reported value is the whole-job rate; under torchrun the reference arm runs on rank 0 only.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_env()
    m = bench.job_max(dist, 10.0 + 5.0 * rank)          # rank 1 is the slow one
    a = bench.parse(["--workload", "spectral", "--grid", "8", "--items", "2", "--increments", "2"])
    Y = bench.gen_stream(a, seed=r)
    digest = float(np.abs(Y).sum())
    d = torch.tensor([digest], dtype=torch.float64)
    g = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(g, d)
    out.put((r, w, lr, m, [float(x) for x in g]))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_job_time_and_own_distinct_streams():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29511
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, (rank, world, local, m, digests) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert m == 15.0                                    # the maximum over ranks on every rank
        assert digests[0] != digests[1]                     # seed = rank: independent streams
    assert bench.job_rate_gbs(1e9, 2, 0.5) == 4.0           # whole-job rate: both ranks' bytes


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", "29512", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "spectral", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--grid", "8", "--items", "2",
           "--increments", "2", "--cpu-seconds", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"

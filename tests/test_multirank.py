"""Multi-process paths of the benchmark, on CPU (world size 2).

Under torchrun every rank counts its own replica library (same shape, its own seed: weak scaling)
with no data-path collective; the job's time is the slowest rank's and its windows are all ranks'
windows. These tests run that reduction on two `gloo` ranks, the reference arm under two ranks
(rank 0 alone runs and prints; the other rank exits 0 without work), and the per-rank libraries.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank r: 10 + r ms per step, 1000 (r + 1) windows; and a second call with one value
        both = bench.reduce_over_ranks([10.0 + rank, 1000 * (rank + 1)], ["max", "sum"], "cpu")
        e2e = bench.reduce_over_ranks([0.5 * (rank + 1)], ["max"], "cpu")
        q.put((rank, both, e2e))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_on_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_reduce_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in procs:
            rank, both, e2e = q.get(timeout=180)
            got[rank] = (both, e2e)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for rank in (0, 1):  # every rank sees the slowest rank's time and the sum of the windows
        assert got[rank] == ([11.0, 3000.0], [1.0])


def test_reduction_without_a_group_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks([1.5, 7], ["max", "sum"], "cpu") == [1.5, 7.0]


def test_reference_arm_under_two_ranks_runs_on_rank_0_only():
    outs = {}
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT="29511")
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                            "--workload", "small", "--scale", "0.02", "--steps", "1", "--warmup", "1",
                            "--cpu-sample-reads", "2000"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[rank] = [l for l in r.stdout.splitlines() if l.strip()]
    assert outs[1] == []  # no work, no output
    assert len(outs[0]) == 1
    line = json.loads(outs[0][0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_each_rank_counts_its_own_replica_library():
    sys.path.insert(0, ROOT)
    import bench

    a, _ = bench.workload("small", 0.01, 0)
    b, _ = bench.workload("small", 0.01, 1)
    assert a.n_reads == b.n_reads and a.bases.size == b.bases.size and a.k == b.k  # same shape
    assert not np.array_equal(a.bases, b.bases)  # different seed

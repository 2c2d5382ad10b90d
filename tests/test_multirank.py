"""The multi-GPU path of bench.py without a GPU: N replicas, one per rank, with no collective on
the data path; the timed region is the slowest rank's, reduced with an all-reduce MAX (NCCL on
the GPUs, here gloo on two CPU ranks), and the whole-job value counts every rank's nodes.  The
reference arm under torchrun runs on rank 0 only and prints one line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = bench.max_over_ranks(values[rank], world, "cpu")
        out.put((rank, ms, bench.job_mlups(1000, 10, world, ms)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [3.5, 7.25]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [7.25, 7.25]
    # 1000 nodes x 10 steps on each of 2 ranks in 7.25 ms
    assert res[0][2] == pytest.approx(2 * 1000 * 10 / 7.25e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0
    assert bench.job_mlups(8, 5, 1, 2.0) == pytest.approx(8 * 5 / 2e-3 / 1e6)


def test_reference_arm_under_torchrun_two_ranks():
    """bench.py --impl reference --gpus 2 under torchrun: rank 0 times the FP64 oracle and prints
    one JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"

"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The path does not shard: N GPUs run N independent replicas, each on its own
query stream, and the job's time is the slowest rank's.  These tests run
that aggregation with two gloo ranks and no GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) seconds: the job took the slowest rank's time
        t_max = bench.max_over_ranks(rank + 1.0, world)
        value = bench.whole_job_value(world, 1024, 3, t_max)
        qs = bench.rank_queries(1000, 8, 2, rank)
        np.savez(f"{out_path}.{rank}.npz", t_max=t_max, value=value, qs=qs)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation(tmp_path):
    port = _free_port()
    out = str(tmp_path / "r")
    tmp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    r0 = np.load(out + ".0.npz")
    r1 = np.load(out + ".1.npz")
    assert float(r0["t_max"]) == 2.0 and float(r1["t_max"]) == 2.0
    assert float(r0["value"]) == pytest.approx(2 * 1024 * 3 / 2.0)
    assert float(r1["value"]) == float(r0["value"])
    # each replica draws its own queries, all inside U
    assert r0["qs"].shape == (2, 8)
    assert not np.array_equal(r0["qs"], r1["qs"])
    assert r0["qs"].max() < 1000 and r1["qs"].max() < 1000


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.whole_job_value(1, 1024, 3, 1.5) == pytest.approx(2048.0)


def _ref_worker(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    import bench
    # the reference arm: rank 0 alone runs the oracle; other ranks do no work
    args = bench.parse(["--impl", "reference", "--graph", "tiny", "--steps", "1",
                      "--warmup", "3", "--cpu-queries", "2"])
    out = bench.run_reference(args, rank, world)
    ok = None
    if out is not None:
        cb, e2e = out["cpu_baseline"], out["e2e"]
        ok = (out["value"] > 0 and out["impl"] == "reference" and out["steps"] == 1 and out["warmup"] == 3
              and cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == out["value"]
              and "rounds" in cb["sample"] and e2e["value"] == out["value"]
              and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0)
    with open(f"{out_path}.{rank}.txt", "w") as f:
        f.write("none" if out is None else repr(ok))


def test_reference_arm_runs_on_rank0_only(tmp_path):
    out = str(tmp_path / "ref")
    tmp.start_processes(_ref_worker, args=(2, 0, out), nprocs=2, join=True, start_method="spawn")
    assert open(out + ".0.txt").read() == "True"
    assert open(out + ".1.txt").read() == "none"

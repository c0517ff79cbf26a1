"""bench.py's multi-rank aggregation (replicas, one per GPU) on CPU ranks over gloo:
the job's time per step is the slowest rank's, and throughput counts every rank's work."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 95.0][rank]           # rank 0 is the slow one
        total = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
        out[rank] = (total, bench.job_throughput(world, 4096, total / 10))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks_and_throughput_sums_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 120.0
    # 10 steps in 120 ms -> 12 ms per step, 2 replicas of 4096 units each
    assert out[0][1] == pytest.approx(2 * 4096 / 0.012)
    assert bench.max_over_ranks(3.5) == 3.5


def test_roofline_traffic_follows_the_kernel_sources(tmp_path):
    """`roofline.traffic` comes from a recorded ncu capture only while the kernel's sources
    hash to the recorded value; any edit makes it null (the counters no longer apply)."""
    import hashlib
    import json
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"dram_bytes_per_launch": 123.0, "sources": ["k.cu"],
                 "source_sha1": hashlib.sha1(src.read_bytes()).hexdigest()}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic("k", root=str(tmp_path)) == 123.0
    assert bench.measured_traffic("other", root=str(tmp_path)) is None
    src.write_text("__global__ void k() { }\n")
    assert bench.measured_traffic("k", root=str(tmp_path)) is None

"""The replica path of bench.py at world size 2 on CPU (gloo): barrier,
max-over-ranks timing and whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    r, w = bench.dist_init("gloo")
    bench.barrier()
    t = bench.max_over_ranks(1.0 + rank)          # rank 1 is the slowest
    v = bench.replica_value(10.0, w, t)
    if r == 0:
        with open(out_path, "w") as fh:
            fh.write(f"{w} {t} {v}")
    bench.barrier()
    dist.destroy_process_group()


def test_replicas_world_size_two(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "out.txt"
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    w, t, v = out.read_text().split()
    assert int(w) == 2 and float(t) == 2.0 and float(v) == pytest.approx(10.0)


def test_single_process_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(8.0, 1, 2.0) == 4.0

"""Host logic of bench.py's multi-replica path on CPU: two gloo ranks agree on the slowest
replica's step time, and the whole-job throughput counts every rank's elements (weak scaling).
The replicas share no data, so this reduction of the timing is the only collective."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, "cpu")   # rank 1 is the slower replica
        td.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(repr(ms))
    finally:
        td.destroy_process_group()


def test_slowest_replica_sets_the_step_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [float((tmp_path / f"rank{r}.txt").read_text()) for r in range(world)]
    assert got == [125.0, 125.0]


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, "cpu") == 42.5


@pytest.mark.parametrize("world", [1, 2, 8])
def test_throughput_counts_every_replica(world):
    sys.path.insert(0, ROOT)
    import bench
    # 4096 elements per replica in 125 ms on the slowest one
    assert bench.replicas_throughput(4096, world, 125.0) == pytest.approx(world * 4096 / 0.125)

"""The multi-rank bench path on CPU (gloo, world size 2): each rank renders
its own poses (no data-path collective), the job's time is the slowest
rank's, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.rank_poses(list(range(64)), rank, world)[:8]
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, torch.device("cpu"))

        class Args:
            pass

        # the reference arm: ranks other than 0 return at once, without work
        skipped = rank != 0 and bench.run_reference(Args(), rank, world) is None
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{','.join(map(str, mine))}\n{ms}\n{int(skipped)}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_poses_and_take_the_slowest_time(tmp_path):
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    lines = [open(tmp_path / f"r{r}.txt").read().split("\n") for r in range(2)]
    poses = [list(map(int, l[0].split(","))) for l in lines]
    assert poses[0] == [0, 2, 4, 6, 8, 10, 12, 14] and poses[1] == [1, 3, 5, 7, 9, 11, 13, 15]
    assert not set(poses[0]) & set(poses[1])
    assert float(lines[0][1]) == float(lines[1][1]) == 15.0  # max over ranks
    assert lines[1][2] == "1"

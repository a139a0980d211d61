"""Replica shards over two ranks (gloo, CPU): each rank simulates its replica
range of one batch with the oracle; together they reproduce the single-process
run exactly, and the throughput figures combine as (sum of events, max time)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1010_2438_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, R_per_rank, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1010_2438_gb300 import shard as S
    from paper_1010_2438_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = W.flat8x12(R=R_per_rank * world)
    off, cnt = S.weak_shard(R_per_rank, rank)
    res = oracle.simulate(b, off, off + cnt)
    hashes = torch.from_numpy(res["hash"].view(np.int64).copy())
    gathered = [torch.zeros_like(hashes) for _ in range(world)]
    dist.all_gather(gathered, hashes)
    ev, tm = S.combine(float(res["events"].sum()), 1.0 + rank, device="cpu")
    if rank == 0:
        np.save(os.path.join(out_dir, "hashes.npy"), torch.cat(gathered).numpy())
        np.save(os.path.join(out_dir, "combined.npy"), np.array([ev, tm]))
    dist.destroy_process_group()


def test_two_rank_shards_reproduce_single_run(tmp_path):
    import oracle
    from paper_1010_2438_gb300 import workloads as W

    world, R = 2, 6
    mp.start_processes(_rank_main, args=(world, _free_port(), R, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    full = oracle.simulate(W.flat8x12(R=R * world))
    got = np.load(tmp_path / "hashes.npy").view(np.uint64)
    assert np.array_equal(got, full["hash"])
    ev, tm = np.load(tmp_path / "combined.npy")
    assert ev == full["events"].sum()
    assert tm == 2.0


def test_shard_ranges():
    assert shard.weak_shard(100, 3) == (300, 100)
    for total, world in ((10, 3), (65536, 8), (7, 7), (5, 8)):
        parts = [shard.strong_shard(total, world, r) for r in range(world)]
        covered = [i for off, cnt in parts for i in range(off, off + cnt)]
        assert covered == list(range(total))

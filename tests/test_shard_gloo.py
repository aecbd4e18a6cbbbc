"""Sharding over ranks: two gloo ranks on CPU each draw their own index range with the
oracle (the product's sharding rule), gather, and must reproduce one single-process
run over the whole range exactly."""
import os

import numpy as np
import torch
import torch.multiprocessing as mp

from paper_2109_07358_gb300.shard import shard_range, step_offset


def test_shard_ranges_partition_the_job():
    for total in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1
    seen = set()
    for step in range(3):
        for r in range(4):
            lo = step_offset(step, r, 4, 10)
            rng = set(range(lo, lo + 10))
            assert not (rng & seen)
            seen |= rng


def _worker(rank, world, port, total, out_path):
    import torch.distributed as dist

    from oracle import ffs_oracle as o
    from paper_2109_07358_gb300 import workloads as w
    from paper_2109_07358_gb300.shard import gather, shard_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = w.haar(12, 4, seed=1)
    lo, hi = shard_range(total, rank, world)
    local = torch.from_numpy(o.sample(U, hi - lo, seed=5, first_sample_index=lo))
    full = gather(local, total)
    if rank == 0:
        np.save(out_path, full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sharding_matches_single_run(tmp_path):
    from oracle import ffs_oracle as o
    from paper_2109_07358_gb300 import workloads as w

    total = 25
    port = 29500 + (os.getpid() % 2000)
    out = str(tmp_path / "x.npy")
    mp.start_processes(_worker, args=(2, port, total, out), nprocs=2, start_method="spawn")
    sharded = np.load(out)
    single = o.sample(w.haar(12, 4, seed=1), total, seed=5)
    assert np.array_equal(sharded, single)

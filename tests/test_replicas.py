"""Multi-rank host logic on CPU (gloo, two processes): work assignment of a
batch to ranks and the whole-job throughput (units of all ranks over the
slowest rank's time) that the benchmark reports for N GPUs."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1601_05527_gb300 import replicas


def test_shard_by_size_partitions_and_balances():
    rng = np.random.default_rng(3)
    sizes = rng.integers(1000, 200_001, size=512)
    for ws in (1, 2, 3, 8):
        parts = [replicas.shard_by_size(sizes, ws, r) for r in range(ws)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [int(sizes[p].sum()) for p in parts]
        # LPT bound: no rank exceeds the average by more than the largest graph
        assert max(loads) - sum(loads) / ws <= sizes.max()
    with pytest.raises(ValueError):
        replicas.shard_by_size(sizes, 2, 2)


def test_single_process_reductions_are_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(10.0, 2.0) == 5.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [5, 9, 2, 7, 7, 1, 3]
        mine = replicas.shard_by_size(sizes, world, rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        seconds = 1.0 + rank               # rank 1 is the slower one
        units = 100.0 * (rank + 1)
        rate = replicas.whole_job_rate(units, seconds)
        slowest = replicas.max_over_ranks(seconds)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([rate, slowest, len(sum(gathered, []))], dtype=np.float64))
        assert sorted(sum(gathered, [])) == list(range(len(sizes)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_aggregation(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        rate, slowest, count = np.load(tmp_path / f"r{r}.npy")
        assert slowest == 2.0
        assert rate == pytest.approx(300.0 / 2.0)
        assert count == 7

"""The N>1 path of the benchmark on CPU: two gloo ranks (no GPU).

The work shards by replicas: every rank runs its own seed, no data crosses
ranks, and the job's time is the slowest rank's (an all-reduce of the elapsed
time with MAX).  Checked here with the same helpers the benchmark uses.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import bench
    import oracle as O

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        elapsed = 1.5 + rank  # the slowest rank decides
        t = bench.max_over_ranks(elapsed, dist)
        st = O.init(64, 64, bench.rank_seed(rank), 0.5)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([[t], st.n.ravel()]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    assert r0[0] == r1[0] == 2.5  # both ranks report the max elapsed time
    assert not np.array_equal(r0[1:], r1[1:])  # independent replicas on each rank


def test_single_process_needs_no_collective():
    import bench

    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.rank_seed(0) != bench.rank_seed(1)

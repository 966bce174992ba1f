"""The multi-GPU path of the benchmark is replicas only: each rank solves its
own right-hand sides and the ranks meet only to take the slowest rank's time.
That host logic runs here on CPU with two gloo ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, outdir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import hisq_inputs as hi
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # the slower rank decides
        t = bench.max_over_ranks(ms, world, torch.device("cpu"))
        val = bench.per_rhs(t, steps=3, n_rhs=4, world=world)
        b = hi.gaussian_sources((2, 2, 2, 2), 4, bench.replica_source_seed(rank))
        np.save(os.path.join(outdir, f"b{rank}.npy"), b)
        with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {val}")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_own_sources(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(world)]
    for t, val in res:
        assert t == 15.0
        assert val == pytest.approx(15.0 / (3 * 4 * world))
    b0, b1 = np.load(tmp_path / "b0.npy"), np.load(tmp_path / "b1.npy")
    assert not np.array_equal(b0, b1)  # independent replicas: different sources


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, None) == 7.5
    assert bench.per_rhs(32.0, steps=2, n_rhs=16, world=1) == 1.0

"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own
independent problems, and the timing reduced to the slowest rank.  The path
shards whole problems across ranks; there is no data exchange to test."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    assert (w, r) == (world, rank)
    # independent problems per rank (a small 2D problem from the same generator)
    from paper_0906_2704_gb300 import synth
    h = synth.gaussian_psf_2d_separable(1.0, 5)
    g, _ = synth.problem_2d(bench.rank_seed(rank), 12, 14, h, 0.01, count=2)
    # slowest rank decides the time; every rank sees the same reduced value
    mine = 0.1 * (rank + 1)
    slowest = bench.max_over_ranks(mine, dist, "cpu")
    rate = bench.whole_job_rate(world, 2, 5, slowest)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([slowest, rate, g.sum()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == pytest.approx(0.2)                  # max over ranks
    assert r0[1] == pytest.approx(world * 2 * 5 / 0.2)            # whole-job images per second
    assert r0[2] != r1[2]                                         # different problems per rank


def test_single_process_needs_no_collective():
    import bench
    assert bench.max_over_ranks(0.37) == 0.37
    assert bench.whole_job_rate(1, 32, 10, 0.5) == 640.0

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


def _shard_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_0906_2704_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    # the uneven batch as the batched workload builds it (count problems per rank)
    count = 96
    items, gs, _ = synth.batch_uneven(7, count * w)
    lo, hi = bench.shard_by_weight([it[0] * it[1] for it in items], w, r)
    mine = np.arange(lo, hi)
    pixels = float(sum(gs[i].size for i in mine))
    # gather every rank's item list and pixel count on every rank (host data only)
    lists = [None] * w
    dist.all_gather_object(lists, (mine.tolist(), pixels))
    np.save(os.path.join(out_dir, f"s{rank}.npy"),
            np.array([len(items), max(p for _, p in lists), min(p for _, p in lists),
                      max(it[0] * it[1] for it in items)], dtype=np.float64))
    with open(os.path.join(out_dir, f"s{rank}.txt"), "w") as fh:
        fh.write(" ".join(str(i) for lst, _ in lists for i in lst))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_uneven_batch_shards_cover_every_problem_once(tmp_path, world):
    """The batched workload's partition under several ranks (unmeasured on hardware:
    one GPU per call here): contiguous shards whose union is the whole batch, each
    problem exactly once, pixel counts balanced to within one problem."""
    mp.start_processes(_shard_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        total, pmax, pmin, biggest = np.load(tmp_path / f"s{r}.npy")
        got = [int(v) for v in (tmp_path / f"s{r}.txt").read_text().split()]
        assert got == list(range(int(total)))              # ordered, complete, no repeats
        assert pmax - pmin <= biggest                      # balanced to within one problem


def test_shard_by_weight_edge_cases():
    import bench
    assert bench.shard_by_weight([5.0], 1, 0) == (0, 1)
    assert bench.shard_by_weight([], 2, 0) == (0, 0) and bench.shard_by_weight([], 2, 1) == (0, 0)
    # more ranks than problems: some shards are empty, none overlap
    cuts = [bench.shard_by_weight([1.0, 1.0], 4, r) for r in range(4)]
    covered = [i for lo, hi in cuts for i in range(lo, hi)]
    assert covered == [0, 1]
    w = np.random.default_rng(3).integers(1, 100, size=257).astype(float)
    cuts = [bench.shard_by_weight(w, 5, r) for r in range(5)]
    assert cuts[0][0] == 0 and cuts[-1][1] == 257
    assert all(cuts[r][1] == cuts[r + 1][0] for r in range(4))

"""The N > 1 host path of bench.py (replicas only, one process per GPU) with world size 2 on the
gloo backend: the barrier, the maximum over ranks of the per-rank time, the whole-job value of
weak-scaled replicas, and the reference arm, which rank 0 alone runs and prints."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    # per-rank times: the job is as slow as its slowest rank
    t = bench.max_over_ranks(0.5 + rank, world)
    value = bench.job_throughput(world, 1000, t)
    bench.barrier(world)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
        json.dump({"t": t, "value": value}, fh)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    mp.spawn(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert res[0]["t"] == res[1]["t"] == 1.5
    assert res[0]["value"] == res[1]["value"] == 2 * 1000 / 1.5


def test_reference_arm_prints_on_rank_zero_only(capsys):
    """Rank 1 of the reference arm does no work and prints nothing."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, gpus = 1, 0, 2

    bench.run_reference(Args, world=2, rank=1)
    assert capsys.readouterr().out == ""


def _shard_worker(rank, world, port, outdir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import synthetic as W

    draws = W.batch_draws(64, seed=4)
    unknowns = [d["mx"] * d["mx"] * d["n"] for d in draws]
    mine = bench.batch_shard(draws, unknowns, world, rank)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    with open(os.path.join(outdir, f"shard{rank}.json"), "w") as fh:
        json.dump({"mine": mine, "parts": parts, "unknowns": unknowns,
                   "thetas": [d["theta"] for d in draws]}, fh)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_partition_over_gloo_ranks(tmp_path, world):
    """The 64-instance batch split over ranks with no collective on the data path: every rank
    computes the same partition on its own, the parts are disjoint and cover every instance, and
    the largest load stays within the greedy bound (total / ranks + largest instance)."""
    import torch.multiprocessing as mp

    from paper_2201_10062_gb300 import shard

    port = _free_port()
    mp.spawn(_shard_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"shard{r}.json")) for r in range(world)]
    parts = res[0]["parts"]
    for r in range(world):
        assert res[r]["parts"] == parts  # the same split on every rank
        assert res[r]["mine"] == parts[r]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))  # complete and disjoint
    costs = [shard.instance_cost(u, t) for u, t in zip(res[0]["unknowns"], res[0]["thetas"])]
    loads = shard.loads(costs, parts)
    assert max(loads) <= sum(costs) / world + max(costs)
    assert all(len(p) > 0 for p in parts)


def test_partition_edge_cases():
    from paper_2201_10062_gb300 import shard

    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5.0], 2) == [[0], []]
    # equal costs spread round-robin by index
    assert shard.partition([1.0] * 4, 2) == [[0, 2], [1, 3]]
    # one rank holds everything
    assert shard.partition([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_bench_roofline_and_update_accounting():
    """Host arithmetic of the bench's roofline: Sec. 8(d)'s bytes (84 per unknown and iteration
    in mixed precision plus 24 per refinement step) over the solve time, and the grouped
    update's bytes per solve (4 per pending z_j and iteration, 48 per launch)."""
    sys.path.insert(0, ROOT)
    import bench

    peak = {"hbm_gbs": 1000.0, "src": "test"}
    r = bench.roofline_iter("mixed", 10**6, 10, 2, 1e-3, peak)
    assert r["achieved"] == pytest.approx((84 * 10 + 24 * 2) * 10**6 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    # 39 iterations in groups of 8: 5 launches; in groups of 1: 39 launches of 4 + 48 B each
    assert bench.update_bytes_per_step(100, 39, 8) == (4 * 39 + 48 * 5) * 100
    assert bench.update_bytes_per_step(100, 39, 1) == 52 * 39 * 100
    prof = {"update": {"launches": 15, "timed": 15, "ms": 3.0},
            "stencil": {"launches": 117, "timed": 117, "ms": 9.0}}
    t = bench.kernel_table(prof, "mixed", 100, 3, peak, iterations=39, group=8)
    assert t["update"]["bytes_per_step"] == (4 * 39 + 48 * 5) * 100
    assert t["update"]["achieved_gbs"] == pytest.approx(t["update"]["bytes_per_step"] / 1e-3 / 1e9)
    assert t["stencil"]["bytes_per_launch"] == 12 * 100
    assert t["update"]["share"] == pytest.approx(0.25)

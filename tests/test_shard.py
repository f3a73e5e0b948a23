"""Sharding the batched encode over ranks: a deterministic cost-balanced
split of independent clips (every clip on exactly one rank), and the
aggregation of the ranks' timings, on two CPU ranks over gloo."""

import os
import socket
import sys

import pytest

from gs2d_inputs import clip_table

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sizes_of(count=32, seed=1000):
    return [(c["width"], c["height"], c["n"]) for c in clip_table(count, seed)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_clip_once_and_balances(world):
    from paper_2505_09324_gb300.shard import clip_cost, partition_clips, shard_loads
    sizes = sizes_of()
    parts = partition_clips(sizes, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))
    assert all(p == sorted(p) for p in parts)
    loads = shard_loads(sizes, parts)
    total, biggest = sum(loads), max(clip_cost(*s) for s in sizes)
    # longest-processing-time first: no rank exceeds the mean by more than one clip
    assert max(loads) <= total / world + biggest
    assert partition_clips(sizes, world) == parts  # deterministic
    if world == 1:
        assert parts == [list(range(len(sizes)))]


def test_partition_edge_cases():
    from paper_2505_09324_gb300.shard import partition_clips
    assert partition_clips([], 3) == [[], [], []]
    assert partition_clips([(10, 10, 1)], 2) == [[0], []]
    # equal costs alternate over the ranks
    assert partition_clips([(8, 8, 4)] * 4, 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        partition_clips([(8, 8, 4)], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2505_09324_gb300.shard import partition_clips
    mine = partition_clips(sizes_of(), world)[rank]
    got = [None] * world
    dist.all_gather_object(got, mine)
    ms, hits = bench.shard_aggregate(1.0 + rank, 100 * (rank + 1), world, "cpu")
    out.put((rank, got, ms, hits))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_batch_and_aggregate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = len(sizes_of())
    for rank, got, ms, hits in res:
        assert sorted(i for part in got for i in part) == list(range(n))
        assert set(got[0]).isdisjoint(got[1])
        assert ms == 2.0 and hits == 300.0   # slowest rank; pairs of both

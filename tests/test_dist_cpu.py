"""The benchmark's multi-rank path (one independent frame per rank, the
slowest rank's time, whole-job throughput) on two CPU ranks over gloo."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    total, value = bench.whole_job(100.0 + 50.0 * rank, 10, world, "cpu")
    # the reference arm: ranks other than 0 leave without work
    ref_rc = bench.run_reference(None) if rank != 0 else 0
    out.put((rank, total, value, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_two_gloo_ranks():
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
    # both ranks see the slowest rank's time; value = time / (steps x ranks)
    assert [r[1] for r in res] == [150.0, 150.0]
    assert all(abs(r[2] - 150.0 / 20) < 1e-12 for r in res)
    assert res[1][3] == 0


def test_whole_job_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(80.0, 8, 1) == (80.0, 10.0)

"""The bench's multi-rank logic (replicas on one node) on CPU processes: two
ranks over gloo, rendezvous on 127.0.0.1.  The job's time is the slowest
rank's; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # rank k reports (k + 1) x 10 ms: every rank sees the maximum
        got = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
        # the reference arm: ranks other than 0 leave without work
        ref = bench.run_reference(None) if rank != 0 else None
        out.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_leave_the_reference_to_rank_0():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g for _, g, _ in res] == [20.0, 20.0]
    assert res[1][2] == 0


def test_single_process_reduction_is_the_value_itself():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5

"""Host logic of bench.py's multi-rank path on CPU: two gloo ranks (127.0.0.1) agree on the
slowest rank's time, and the CPU-oracle reference arm does its work on rank 0 only."""
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


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks_of(1.5 + rank, world, torch.device("cpu"))
        r, lr, w = bench.dist_env()
        # the reference arm returns immediately on ranks other than 0
        ran = None
        if rank != 0:
            class A:  # minimal argument object
                steps, warmup, gpus = 1, 0, world
            bench.run_reference(A())
            ran = "skipped"
        q.put((rank, t, (r, lr, w), ran))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [2.5, 2.5]
    assert out[0][2] == (0, 0, 2) and out[1][2] == (1, 1, 2)
    assert out[1][3] == "skipped"

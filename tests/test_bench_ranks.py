"""Host logic of bench.py's multi-rank path (replicas), on CPU with gloo, world size 2."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank times its own replica; the job time is the slowest rank
    t = bench._over_ranks([10.0 + rank, 3.0 * (rank + 1)], dist, "cpu")
    n = bench._over_ranks([7.0 * (rank + 1)], dist, "cpu", op="sum")
    q.put((rank, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
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
    for rank, t, n in out:
        assert t == [11.0, 6.0] and n == [21.0]


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._over_ranks([1.5, 2], None, "cpu") == [1.5, 2.0]

"""The bench's multi-rank path on CPU: two gloo ranks, no GPU.

Each rank runs an independent replica (weak scaling, no collective on the data
path); the only collectives are the barrier and the maximum of the timed region over
ranks, and the reported value is the updates of all ranks over that maximum.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    t_local = 100.0 + 50.0 * rank               # rank 1 is the slower one
    t_max = bench.dist_max(dist, t_local, "cpu")
    dist.barrier()
    q.put((rank, t_max, bench.aggregate_mlups(1_000_000, t_max, world)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_throughput():
    torch = pytest.importorskip("torch")
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    # 2 ranks x 1e6 updates over 0.15 s
    assert all(abs(o[2] - 2e6 / 0.15 / 1e6) < 1e-9 for o in out)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(None, 3.5, "cpu") == 3.5
    assert bench.aggregate_mlups(2_000_000, 1000.0, 1) == 2.0

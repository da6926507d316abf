"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
replica, a barrier around the timed region and the maximum of the per-rank
times (weak scaling: no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(w)
    t = bench.allmax(w, 1.0 + rank)            # rank-dependent "elapsed time"
    case = bench.make_case("advection_20", replica=r)
    out[rank] = (t, int(case.mesh.nodes.sum() * 1e6))
    dist.destroy_process_group()


def test_two_rank_barrier_and_max():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 2.0        # every rank sees the slowest rank's time
    assert out[0][1] != out[1][1]               # each rank owns a different replica (seed + rank)

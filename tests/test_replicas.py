"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas only.

The sweep does not exchange data between GPUs here (each rank runs its own
lattices), so the only cross-rank steps are the barrier and the max-over-
ranks timing that turn per-rank times into one whole-job number.
"""
import os
import socket

import pytest

import bench

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_info()
    dist.barrier()
    t = bench.max_over_ranks(1.5 + rank)       # per-rank seconds
    v = bench.replica_value(3.0e9, w, t)       # 3e9 updates per rank
    out.put((r, w, local, t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_max_time_and_sum_of_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, t, v) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert t == 2.5                           # the slower rank's time
        assert v == pytest.approx(2 * 3.0e9 / 2.5e9)


def test_single_process_is_identity():
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.replica_value(1e9, 1, 1.0) == pytest.approx(1.0)

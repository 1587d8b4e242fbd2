"""The bench's multi-rank aggregation on CPU (gloo, world size 2).

Every rank maps its own map (weak scaling, no data exchange); the only
collectives are the barrier and the max over ranks of the timings.
"""

import os
import socket

import pytest
import torch
import torch.distributed as td
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        td.barrier()
        my_ms = [120.0, 180.0][rank]              # rank 1 is the slow one
        m = bench.max_over_ranks(my_ms)
        v = bench.whole_job_mpix_s(4096.0 * 4096, 100, world, m)
        q.put((rank, m, v))
    finally:
        td.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 180.0
        assert v == pytest.approx(2 * 4096 * 4096 * 100 / 0.180 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_mpix_s(1e6, 10, 1, 1000.0) == pytest.approx(10.0)

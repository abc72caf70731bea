"""CPU, two ranks over gloo: the host side of the multi-GPU runs -- every
rank takes its own block of units (weak scaling, no collective on the data
path) and the job's time is the maximum, its bytes the sum, over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        own = bench.shard_units(5, ws, rank)
        mx = bench.reduce_over_ranks([1.0 + rank, 7.0 - 3 * rank], "max")
        sm = bench.reduce_over_ranks([float(len(own)), 0.5], "sum")
        q.put((rank, env, own, mx, sm))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in procs:
            rank, env, own, mx, sm = q.get(timeout=180)
            res[rank] = (env, own, mx, sm)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert res[0][0] == (2, 0, 0) and res[1][0][:2] == (2, 1)
    units = res[0][1] + res[1][1]
    assert sorted(units) == list(range(10)) and not set(res[0][1]) & set(res[1][1])
    for r in (0, 1):
        assert res[r][2] == [2.0, 7.0]
        assert res[r][3] == [10.0, 1.0]


def test_one_process_is_the_identity():
    import bench

    assert bench.shard_units(4, 1, 0) == [0, 1, 2, 3]
    assert bench.reduce_over_ranks([3.0, 4.5], "max") == [3.0, 4.5]

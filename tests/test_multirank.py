"""The multi-process path of bench.py on CPU: two replicas over gloo.

bench.py runs one independent replica per GPU (the operator needs no data
exchange, so there is no collective on the data path); the only cross-rank
steps are the barriers around the timed region and the max over ranks of its
time.  These tests run those steps in two spawned processes with the gloo
backend on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.ranks_barrier(world)
        job_ms = bench.max_over_ranks(local_ms[rank], world)
        bench.ranks_barrier(world)
        q.put((rank, job_ms, bench.job_value(world, 8, job_ms)))
    finally:
        dist.destroy_process_group()


def _run(world, local_ms):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, local_ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    for p in procs:
        assert p.exitcode == 0
    out = {}
    while not q.empty():
        rank, ms, val = q.get()
        out[rank] = (ms, val)
    return out


def test_two_replicas_take_the_slowest_time():
    out = _run(2, [0.35, 0.42])
    assert sorted(out) == [0, 1]
    for rank in (0, 1):
        ms, val = out[rank]
        assert ms == pytest.approx(0.42)
        # weak scaling: both replicas' batches count
        assert val == pytest.approx(2 * 8 / 0.42e-3)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.job_value(1, 8, 0.5) == pytest.approx(16000.0)

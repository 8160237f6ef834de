"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2,
127.0.0.1 rendezvous) with different local times agree on the max-over-ranks
time and on the whole-job (weak-scaling) rate; a single process without a
process group reduces to itself."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, ws, port, local_times, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(local_times[rank], device="cpu")
        rate = bench.whole_job_rate(1000.0, ws, t)
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_rate():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    local_times = [0.5, 2.0]
    procs = [ctx.Process(target=_rank, args=(r, ws, port, local_times, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, rate in out:
        assert t == 2.0
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_single_process_reduces_to_itself():
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0

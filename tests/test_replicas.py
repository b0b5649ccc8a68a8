"""Replica bookkeeping across ranks, run as two gloo processes on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_12616_gb300.replicas import aggregate_rate, id_offset, max_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = max_over_ranks(10.0 + 5.0 * rank)
        off = id_offset(rank, 1000)
        out.put((rank, ms, off))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_ids():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]          # every rank sees the slowest time
    assert [r[2] for r in res] == [0, 1000]             # disjoint particle ids


def test_single_process_and_rate():
    assert max_over_ranks(7.5) == 7.5
    assert aggregate_rate(1e6, 4, 500.0) == 8e6
    with pytest.raises(ValueError):
        id_offset(5, 2 ** 30)

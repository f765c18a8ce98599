"""The multi-GPU forms on CPU: LPT sharding of independent units and the
two reductions used across ranks, run as world_size-2 gloo process groups on
127.0.0.1 (no GPU), plus a rank that leaves early being detected on the host
by a short process-group timeout."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2405_07898_gb300 import sharding


def test_lpt_shards_cover_and_balance():
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(1024), np.log(16384), size=512)).astype(int).tolist()
    for nranks in (1, 2, 3, 8):
        shards = sharding.lpt_shards(sizes, nranks)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)
        assert sharding.lpt_shards(sizes, nranks) == shards  # deterministic
        for s in shards:
            assert [sizes[i] for i in s] == sorted((sizes[i] for i in s), reverse=True)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    try:
        if mode == "reduce":
            m = sharding.reduce_max(1.5 + rank)
            v = sharding.allreduce_sum(np.array([float(rank), 1.0, 2.0 ** -40]))
            shards = sharding.lpt_shards([5, 3, 8, 1, 9, 2], world)
            mine = sum([5, 3, 8, 1, 9, 2][i] for i in shards[rank])
            total = sharding.allreduce_sum(np.array([mine]))
            out.put((rank, m, v.tolist(), float(total[0])))
        elif mode == "leave":
            if rank == 1:
                return  # leaves between steps, before the collective
            try:
                sharding.reduce_max(1.0)
                out.put((rank, "no error"))
            except Exception as e:  # the collective times out on the host
                out.put((rank, type(e).__name__))
    finally:
        if mode == "reduce" or rank == 0:
            try:
                dist.destroy_process_group()
            except Exception:
                pass


def _run(mode, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    for p in procs:
        if p.is_alive():
            p.kill()
    res = []
    while not q.empty():
        res.append(q.get())
    return sorted(res)


def test_two_rank_reductions_gloo():
    res = _run("reduce")
    assert len(res) == 2
    for rank, m, v, total in res:
        assert m == 2.5
        assert v == [1.0, 2.0, 2.0 * 2.0 ** -40]
        assert total == 28.0


def test_rank_that_leaves_is_detected_on_host():
    res = _run("leave")
    assert len(res) == 1 and res[0][0] == 0
    assert res[0][1] != "no error"

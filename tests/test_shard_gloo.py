"""The multi-process path on CPU (gloo, world size 2): stacks split over two
ranks give, stack by stack, the densities, fluxes and ledgers of one process
that runs them all (the streams depend on the global stack index only); the
timing reduction takes the largest time and the sum of the counts."""
import os
import socket

import numpy as np
import pytest

from paper_1807_04733_gb300 import shard
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")


def small_batched():
    return W.batched(n_stacks=5, scale=2e-4, n_steps=40, flags=W.FLAG_DETERMINISTIC)


def run_stacks(wl, lo, hi):
    from oracle.oracle import OracleSim
    out = {}
    for s in range(lo, hi):
        sim = OracleSim(wl, stack=s)
        assert sim.step(wl.n_steps) == 0
        n, J, led = sim.moments()
        out[s] = (n, J, led)
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = small_batched()
        lo, hi = shard.stack_range([st.n0 for st in wl.stacks], rank, world)
        mine = run_stacks(wl, lo, hi)
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        ms, cnt = shard.reduce_measurement(10.0 * (rank + 1), 100.0 + rank, dist)
        if rank == 0:
            merged = {}
            for p in parts:
                merged.update(p)
            q.put((merged, ms, cnt, [shard.stack_range([st.n0 for st in wl.stacks], r, world)
                                     for r in range(world)]))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_one_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, ms, cnt, ranges = q.get(timeout=300)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    wl = small_batched()
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == len(wl.stacks)
    assert ranges[0][1] > 0 and ranges[1][1] > ranges[1][0]
    ref = run_stacks(wl, 0, len(wl.stacks))
    assert sorted(merged) == sorted(ref)
    for s, (n, J, led) in ref.items():
        n2, J2, led2 = merged[s]
        assert led == led2 and np.array_equal(n, n2) and np.array_equal(J, J2)
    assert ms == 20.0 and cnt == 201.0


def test_stack_range_balances_and_covers():
    w = [5, 1, 1, 1, 10, 2, 2, 2, 2, 30]
    for world in (1, 2, 3, 4, 7):
        rs = [shard.stack_range(w, r, world) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == len(w)
        for a, b in zip(rs, rs[1:]):
            assert a[1] == b[0]
    rs = [shard.stack_range([1] * 64, r, 4) for r in range(4)]
    assert [b - a for a, b in rs] == [16, 16, 16, 16]

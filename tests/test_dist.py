"""The multi-rank path on CPU: world size 2 over gloo.

Each rank solves its shard of a scenario batch (with the oracle, since this
host has no GPU), the shards are gathered, and the result must equal the
single-process solve of the whole batch; the timing and count reductions
must give the max and the sum.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

from paper_2605_14103_gb300 import dist as D    # noqa: E402


def test_shard_range_covers_every_scenario_once():
    for B in (0, 1, 7, 128, 4097):
        for world in (1, 2, 3, 8):
            got = [D.shard_range(B, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == B
            for (a, b), (c, d) in zip(got, got[1:]):
                assert b == c
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import zbus_oracle as O
        from paper_2605_14103_gb300 import feeders as F
        f, Sw, Sd, w = F.make_workload("feeder13_b8", B=11)
        lo, hi = D.shard_range(11, rank, world)
        r = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack,
                        Sw[lo:hi], Sd[lo:hi])
        V = torch.from_numpy(r["V"])
        it = torch.from_numpy(r["iters"].astype(np.int64))
        Vall = D.gather_shards(V, 11)
        itall = D.gather_shards(it, 11)
        tmax = D.reduce_max(1.0 + rank)
        tsum = D.reduce_sum(float(hi - lo))
        if rank == 0:
            full = O.solve_coo(f.n_total, f.Y_row, f.Y_col, f.Y_val, f.slack_idx, f.v_slack,
                               Sw, Sd)
            out.put((np.abs(Vall.numpy() - full["V"]).max(),
                     bool(np.array_equal(itall.numpy(), full["iters"])), tmax, tsum))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_gather_equal_the_whole_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs)
    dv, iters_equal, tmax, tsum = q.get(timeout=10)
    assert dv <= 1e-13 and iters_equal
    assert tmax == 2.0 and tsum == 11.0

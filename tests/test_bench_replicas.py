"""The N>1 path of bench.py on CPU: two gloo ranks rendezvous on 127.0.0.1,
pass the barrier, and agree on the maximum time over ranks, from which the
whole-job value is formed (replicas, no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), PNOP_BENCH_GLOO="1")
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    ms = 100.0 * (r + 1)  # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, w)
    q.put((r, w, mx, bench.aggregate_value(100, 5, w, mx)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, mx, val in got:
        assert w == 2 and mx == 200.0
        assert abs(val - 100 * 5 * 2 / 0.2) < 1e-9

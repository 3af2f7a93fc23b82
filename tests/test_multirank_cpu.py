"""The N > 1 bench path on CPU: two gloo ranks, independent replicas, max-over-ranks time.

Streams are independent units, so ranks share nothing but the final timing reduction
(no data-path collective); each rank draws its own stream (rank-keyed seed).
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, dist, "cpu")
    wl = dict(width=16, bands=8, lines=70, batch=70)
    sc, lines = bench.make_inputs(wl, rank)
    dist.barrier()
    q.put((rank, ms, bench.weak_value(1000, world, ms), int(lines.sum()), float(sc.gain[0])))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_draw_distinct_streams():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, sum0, g0), (r1, ms1, v1, sum1, g1) = out
    assert ms0 == ms1 == 15.0                          # max over ranks
    assert v0 == v1 == pytest.approx(1000 * 2 / 0.015)  # whole-job value from the slowest rank
    assert sum0 != sum1 and g0 != g1                   # rank-seeded, independent streams

"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): per-rank
batches of the same shape and the whole-job reduction (slowest rank's time,
all ranks' loadflows)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_2501_17529_b300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.workload(2, n_topo=32)
        topo = bench.rank_topologies(w, 2, 32, rank)
        t, lf = bench.reduce_over_ranks(0.5 + rank, 1000.0 * (rank + 1), "cpu")
        q.put((rank, t, lf, np.asarray(topo.split_sub).tolist(), int(topo.n_topo)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_and_shard():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, lf0, subs0, n0), (r1, t1, lf1, subs1, n1) = out
    assert t0 == t1 == pytest.approx(1.5)          # the slowest rank
    assert lf0 == lf1 == pytest.approx(3000.0)      # all ranks' loadflows
    assert n0 == n1 == 32
    assert subs0 != subs1                            # independent batches of one shape

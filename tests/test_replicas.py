"""The N > 1 path on CPU ranks: world size 2 over gloo (127.0.0.1).  Each
rank runs the FP64 oracle on its own replica rows (the same work a GPU
replica does), and the timing protocol (barrier, max over ranks, whole-job
throughput) and the row partition are checked."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2301_05451_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.env()
    assert (r, w, lr) == (rank, world, rank)
    import oracle
    from paper_2301_05451_gb300 import workloads as W
    spec, params, inputs = W.qnn12(batch=8)
    lo, hi = replicas.row_range(8, rank, world)
    vals = oracle.expvals(spec, W.resolve_angles(spec, params, inputs[lo:hi], batch=hi - lo), nthreads=1)
    dist.barrier()
    secs = 1.0 + rank  # rank 1 is the slow one
    t = replicas.max_over_ranks(secs, dist)
    thr = replicas.aggregate_throughput(10, secs, dist)
    # gather every rank's rows to rank 0 for the check
    import torch
    buf = [torch.zeros(4, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(buf, torch.as_tensor(vals[:, 0], dtype=torch.float64))
    if rank == 0:
        out.put((t, thr, np.concatenate([b.numpy() for b in buf])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo(orc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, thr, rows = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 2.0                      # the slowest rank's time
    assert abs(thr - 10 * 2 / 2.0) < 1e-12  # all ranks' units over the max time
    from paper_2301_05451_gb300 import workloads as W
    spec, params, inputs = W.qnn12(batch=8)
    ref = orc.expvals(spec, W.resolve_angles(spec, params, inputs))[:, 0]
    np.testing.assert_allclose(rows, ref, atol=0, rtol=0)  # the partition covers every row once


def test_row_range_partitions():
    for n in (0, 1, 7, 8, 65):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = replicas.row_range(n, r, world)
                seen.extend(range(lo, hi))
            assert seen == list(range(n))

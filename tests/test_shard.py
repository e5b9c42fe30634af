"""Slice sharding over ranks (Sec. 3.2.3) on CPU ranks: world size 2 over
gloo (127.0.0.1).  Each rank contracts its contiguous share of the slices of
an amplitude network with the FP64 oracle (its loop-nest contraction, with
the sliced wires fixed by projectors), and one FP64 all-reduce adds the
partials; the sum must equal the unsliced amplitude.  The partition itself
is checked for every (units, world) combination."""
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2301_05451_gb300 import shard
from paper_2301_05451_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_values.json")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cases():
    """(name, circuit, angles row, cuts): the 5x5 depth-8 U3/CZ grid with two
    cut wires (4 slices) and the 4x4 one with three (8 slices)."""
    out = []
    for rows, cuts in ((5, [(12, 100), (7, 60)]), (4, [(5, 40), (6, 41), (9, -1)])):
        c, p, _ = W.grid_u3cz(seed=1004, rows=rows, cols=rows, depth=8)
        out.append(("%dx%d" % (rows, rows), c, W.resolve_angles(c, p)[0], cuts))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    res = {}
    for name, c, ang, cuts in _cases():
        seen = []

        def contract_range(first, count):
            seen.extend(range(first, first + count))
            part = sum((oracle.sliced_amplitudes(c, ang, cuts, s, method="tn")[0] for s in range(first, first + count)),
                       0j)
            return torch.tensor([part.real, part.imag], dtype=torch.float64)

        tot = shard.run_sliced(contract_range, 1 << len(cuts), dist)
        res[name] = (complex(tot[0].item(), tot[1].item()), seen)
    q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slice_sharding_gloo(orc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    gold = json.load(open(GOLDEN))["grid_u3cz_5x5_d8"]["1004"]
    for name, c, ang, cuts in _cases():
        ref = complex(*gold) if name == "5x5" else orc.amplitudes(c, ang[None])[0, 0]
        n = 1 << len(cuts)
        # every rank holds the same full sum; each slice was contracted once
        assert got[0][name][0] == got[1][name][0]
        assert sorted(got[0][name][1] + got[1][name][1]) == list(range(n))
        assert abs(got[0][name][0] - ref) <= 1e-4 * abs(ref), (name, got[0][name][0], ref)


def test_share_partitions():
    for n in (0, 1, 2, 7, 8, 65, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [shard.share(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, _) in zip(parts, parts[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.share(4, 2, 2)


def test_allreduce_single_process_packs_fp64():
    v = torch.tensor([[1.5, 2.0]], dtype=torch.float64)
    g = torch.tensor([[0.25, -1.0, 3.0]], dtype=torch.float32)
    sv, sg = shard.allreduce_sum(None, v, g)
    assert sv.dtype == torch.float64 and sg.dtype == torch.float64
    assert sv.shape == v.shape and sg.shape == g.shape
    np.testing.assert_array_equal(sg.numpy(), g.double().numpy())

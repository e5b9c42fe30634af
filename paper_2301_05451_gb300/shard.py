"""Slice and row sharding over ranks (Sec. 3.2.3).

Slicing fixes the values of a few indices of the network; every assignment
gives a sub-network of the same shape, the sub-networks are independent, and
the value of the whole network is the sum of theirs.  Rows of a batch are
independent as well.  So N ranks each take a contiguous share of the slices
(or rows), contract it, and one all-reduce (sum) in FP64 adds the partial
amplitudes or expectation values -- and the partial gradients, which are
sums over slices too.  No other exchange is needed.

`share` is the partition, `allreduce_sum` the one collective, `run_sliced`
puts them together around any function that contracts a slice range, and
`ShardedTreeExec` does so for a compiled tree plan on the rank's GPU
(tdq_exec_set_slice_range).
"""
from __future__ import annotations

import torch


def share(n_units, rank, world):
    """Contiguous share [lo, hi) of n_units for `rank` of `world`: the first
    n_units % world ranks take one unit more, so shares differ by at most one
    and cover every unit once, in order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    base, extra = divmod(int(n_units), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_sum(dist, *parts):
    """The sum over ranks of each tensor in parts, in FP64, with one
    all-reduce (the parts are packed into one buffer on the first part's
    device).  dist = None: a single process, the parts as FP64."""
    flat = [p.reshape(-1).to(torch.float64) for p in parts]
    sizes = [f.numel() for f in flat]
    buf = torch.cat(flat) if flat else torch.zeros(0, dtype=torch.float64)
    if dist is not None and dist.get_world_size() > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    out, o = [], 0
    for p, n in zip(parts, sizes):
        out.append(buf[o:o + n].reshape(p.shape))
        o += n
    return out


def run_sliced(contract_range, n_slices, dist=None):
    """This rank's share of n_slices contracted by contract_range(first,
    count) -> tensor or tuple of tensors (partial sums over those slices),
    then summed over ranks.  Returns the full sums (FP64), on every rank."""
    rank = dist.get_rank() if dist is not None else 0
    world = dist.get_world_size() if dist is not None else 1
    lo, hi = share(n_slices, rank, world)
    parts = contract_range(lo, hi - lo)
    if isinstance(parts, torch.Tensor):
        return allreduce_sum(dist, parts)[0]
    return allreduce_sum(dist, *parts)


class ShardedTreeExec:
    """A compiled tree plan whose slices are shared out over the ranks of a
    process group: each rank contracts its contiguous share of the plan's
    2^n_sliced slices on its own GPU, and one FP64 all-reduce adds the
    partial values (and gradients)."""

    def __init__(self, tree_exec, n_slices, dist=None):
        self.E = tree_exec
        self.dist = dist
        rank = dist.get_rank() if dist is not None else 0
        world = dist.get_world_size() if dist is not None else 1
        self.lo, self.hi = share(n_slices, rank, world)
        self.E.set_slice_range(self.lo, self.hi - self.lo)

    def alloc_outputs(self):
        return self.E.alloc_outputs()

    def run(self, params, inputs=None, values=None, grads=None):
        """Values (FP64) and gradients (FP64, or None) of the whole network."""
        v, g = self.E.run(params, inputs, values=values, grads=grads)
        if g is None:
            return allreduce_sum(self.dist, v)[0], None
        return tuple(allreduce_sum(self.dist, v, g))

    def __getattr__(self, name):  # work(), config(), launches(), status() ... of the rank's exec
        return getattr(self.E, name)

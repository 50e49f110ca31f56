"""Multi-process form of the quadrature: grid blocks are independent work
units (paper Sec. III-E), so ranks evaluate disjoint block ranges and the
single exchange step is a sum of the partial V_xc and E_xc.  Two ways to hand
out the blocks: a static partition balanced by the retained-list work
(partition_blocks), or dynamic pulling of fixed-size chunks from a counter
shared through the torch.distributed store (BlockQueue), the paper's runtime
for heterogeneous grid-batch tasks.

Host logic only (partitioning and the reduction through torch.distributed);
every rank's evaluation runs in the library's kernels.  One GPU per process;
with one GPU per box the hot path runs as replicas, and this module is
exercised by CPU (gloo) ranks in the tests.
"""
from __future__ import annotations

import numpy as np


def block_weights(blk_ptr, bmax=None):
    """Work estimate per grid block from its retained list: n_g^2 (the
    density and V products both scale with the square of the retained
    basis blocks)."""
    n = np.diff(np.asarray(blk_ptr, dtype=np.int64))
    return (n * n).astype(np.float64)


def partition_blocks(weights, world: int):
    """Contiguous grid-block ranges [(g0, g1)] per rank with nearly equal total
    weight: rank r takes the blocks whose cumulative weight midpoint falls in
    [r W / world, (r + 1) W / world).  Ranges are disjoint, ordered, cover all
    blocks, and may be empty when there are fewer blocks than ranks."""
    w = np.asarray(weights, dtype=np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    nb = w.size
    if nb == 0:
        return [(0, 0)] * world
    total = w.sum()
    if total <= 0.0:
        w = np.ones(nb)
        total = float(nb)
    mid = np.cumsum(w) - 0.5 * w
    owner = np.minimum((mid * world / total).astype(np.int64), world - 1)
    bounds = np.searchsorted(owner, np.arange(world + 1), side="left")
    bounds[-1] = nb
    return [(int(bounds[r]), int(bounds[r + 1])) for r in range(world)]


def reduce_exc(V, E, group=None):
    """Sum the ranks' partial V and E in place (torch tensors; gloo for CPU
    tensors, NCCL for CUDA tensors)."""
    import torch.distributed as dist
    dist.all_reduce(V, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(E, op=dist.ReduceOp.SUM, group=group)
    return V, E


def exc_sharded(plan, xc, D, V, E, rank: int, world: int, group=None):
    """This rank's share of kldi_exc followed by the reduction: the plan is
    restricted to the rank's block range (balanced by block_weights), V and E
    (device tensors) receive the full result on every rank."""
    from . import kldi
    ptr, _, _ = plan.lists()
    g0, g1 = partition_blocks(block_weights(ptr), world)[rank]
    plan.set_block_range(g0, g1)
    kldi.exc(plan, xc, D, V, E)
    return reduce_exc(V, E, group)


def reduce_grad(G, E, group=None):
    """Sum the ranks' partial nuclear gradients (natm x 3) and E_xc in place."""
    import torch.distributed as dist
    dist.all_reduce(G, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(E, op=dist.ReduceOp.SUM, group=group)
    return G, E


def exc_grad_sharded(plan, xc, D, G, E, rank: int, world: int, group=None):
    """This rank's share of kldi_exc_grad (its balanced block range) followed by
    the reduction: G and E (device tensors) receive the full result on every
    rank.  The gradient is a sum over grid blocks like E_xc, so the partials add."""
    from . import kldi
    ptr, _, _ = plan.lists()
    g0, g1 = partition_blocks(block_weights(ptr), world)[rank]
    plan.set_block_range(g0, g1)
    kldi.exc_grad(plan, xc, D, G, E)
    return reduce_grad(G, E, group)


class BlockQueue:
    """Dynamic pull scheduler: chunk c covers grid blocks [c chunk, min((c + 1)
    chunk, nblocks)); ranks take the next chunk with one atomic Store.add, so
    every chunk goes to exactly one rank and faster ranks take more.  `key`
    names the counter; use a fresh key per evaluation (the store keeps it)."""

    def __init__(self, store, nblocks: int, chunk: int, key: str):
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.store, self.nblocks, self.chunk, self.key = store, int(nblocks), int(chunk), key

    def take(self):
        c = int(self.store.add(self.key, 1)) - 1
        g0 = c * self.chunk
        if g0 >= self.nblocks:
            return None
        return g0, min(g0 + self.chunk, self.nblocks)


def exc_pulled(plan, xc, D, V, E, queue: BlockQueue, group=None):
    """kldi_exc over the chunks this rank pulls from `queue`, summed, then the
    sum-reduce over ranks (device tensors V, E receive the full result).
    Returns the block ranges this rank evaluated; the plan is left on all its
    grid blocks.  Without an initialised process group of more than one rank
    there is nothing to reduce."""
    import torch
    from . import kldi
    Vp = torch.zeros_like(V)
    Ep = torch.zeros_like(E)
    V.zero_()
    E.zero_()
    done = []
    while True:
        r = queue.take()
        if r is None:
            break
        plan.set_block_range(*r)
        kldi.exc(plan, xc, D, Vp, Ep)
        V += Vp
        E += Ep
        done.append(r)
    plan.set_block_range(0, plan.stats["nblocks"])
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        reduce_exc(V, E, group)
    return done

"""Multi-process form of the quadrature: grid blocks are independent work
units (paper Sec. III-E), so ranks evaluate disjoint block ranges and the
single exchange step is a sum of the partial V_xc and E_xc.

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

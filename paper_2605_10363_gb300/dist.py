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

import pickle
import time

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


def _sum_in_rank_order(t, group=None):
    """Every rank's t gathered and added in rank order, ((t_0 + t_1) + t_2) + ...,
    into t on every rank: the same bits on every rank and in every run, and the
    bits of one process that adds the same partials in that order."""
    import torch.distributed as dist
    parts = [t.new_empty(t.shape) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t.contiguous(), group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    t.copy_(acc)
    return t


def reduce_exc(V, E, group=None, ordered=False):
    """Sum the ranks' partial V and E in place (torch tensors; gloo for CPU
    tensors, NCCL for CUDA tensors).  ordered: add the partials in rank order
    (all-gather, world x the memory of V) so the result does not depend on the
    collective's internal summation order."""
    import torch.distributed as dist
    if ordered:
        return _sum_in_rank_order(V, group), _sum_in_rank_order(E, group)
    dist.all_reduce(V, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(E, op=dist.ReduceOp.SUM, group=group)
    return V, E


def exc_sharded(plan, xc, D, V, E, rank: int, world: int, group=None, ordered=False):
    """This rank's share of kldi_exc followed by the reduction: the plan is
    restricted to the rank's block range (balanced by block_weights), V and E
    (device tensors) receive the full result on every rank."""
    from . import kldi
    ptr, _, _ = plan.lists()
    g0, g1 = partition_blocks(block_weights(ptr), world)[rank]
    plan.set_block_range(g0, g1)
    kldi.exc(plan, xc, D, V, E)
    return reduce_exc(V, E, group, ordered)


def reduce_grad(G, E, group=None, ordered=False):
    """Sum the ranks' partial nuclear gradients (natm x 3) and E_xc in place
    (ordered: in rank order, as in reduce_exc)."""
    import torch.distributed as dist
    if ordered:
        return _sum_in_rank_order(G, group), _sum_in_rank_order(E, group)
    dist.all_reduce(G, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(E, op=dist.ReduceOp.SUM, group=group)
    return G, E


def exc_grad_sharded(plan, xc, D, G, E, rank: int, world: int, group=None, ordered=False):
    """This rank's share of kldi_exc_grad (its balanced block range) followed by
    the reduction: G and E (device tensors) receive the full result on every
    rank.  The gradient is a sum over grid blocks like E_xc, so the partials add."""
    from . import kldi
    ptr, _, _ = plan.lists()
    g0, g1 = partition_blocks(block_weights(ptr), world)[rank]
    plan.set_block_range(g0, g1)
    kldi.exc_grad(plan, xc, D, G, E)
    return reduce_grad(G, E, group, ordered)


class BlockQueue:
    """Dynamic pull scheduler: chunk c covers grid blocks [c chunk, min((c + 1)
    chunk, nblocks)); ranks take the next chunk with one atomic Store.add, so
    every chunk goes to exactly one rank and faster ranks take more.  `key`
    names the counter; use a fresh key per evaluation (the store keeps it).

    With ``lease_timeout`` (seconds) the chunks are leases: taking a chunk
    records its owner, and a rank publishes its cumulative partial result with
    the list of chunks it covers (``publish``) after each chunk.  A rank that
    leaves between chunks, announced (``leave``) or silent (no take or publish
    for ``lease_timeout`` seconds; the ranks share one clock), loses the chunk
    it holds: once the counter is exhausted, ``take`` re-offers every chunk
    that is neither published nor held by a live rank, and returns None only
    when every chunk is published.  ``reduce_published`` then sums the
    published partials, which cover every chunk exactly once."""

    def __init__(self, store, nblocks: int, chunk: int, key: str, rank: int = 0, lease_timeout=None,
                 poll: float = 0.05):
        if chunk < 1:
            raise ValueError("chunk must be >= 1")
        self.store, self.nblocks, self.chunk, self.key = store, int(nblocks), int(chunk), key
        self.rank, self.lease_timeout, self.poll = int(rank), lease_timeout, poll
        self.nchunks = -(-self.nblocks // self.chunk)
        self.mine = []                       # chunks this rank published

    def _range(self, c):
        return c * self.chunk, min((c + 1) * self.chunk, self.nblocks)

    def _k(self, *parts):
        return "/".join([self.key] + [str(p) for p in parts])

    def _beat(self):
        if self.lease_timeout is not None:
            self.store.set(self._k("hb", self.rank), repr(time.time()))

    def _gone(self, r: int) -> bool:
        if self.store.check([self._k("left", r)]):
            return True
        if not self.store.check([self._k("hb", r)]):
            return False
        return time.time() - float(self.store.get(self._k("hb", r)).decode()) > self.lease_timeout

    def _record(self, r: int):
        if not self.store.check([self._k("part", r)]):
            return None
        return pickle.loads(self.store.get(self._k("part", r)))

    def take(self):
        self._beat()
        c = int(self.store.add(self.key, 1)) - 1
        if c < self.nchunks:
            if self.lease_timeout is not None:
                self.store.set(self._k("owner", c), str(self.rank))
            return self._range(c)
        if self.lease_timeout is None:
            return None
        # counter exhausted: re-offer the chunks of ranks that left
        unowned = {}                            # chunk -> first time seen without an owner
        while True:
            pending = False
            for c in range(self.nchunks):
                if self.store.check([self._k("done", c)]):
                    continue
                if not self.store.check([self._k("owner", c)]):
                    # taken from the counter, owner not yet recorded; if it stays
                    # so for a lease, the taker left in between: claim it
                    t0 = unowned.setdefault(c, time.time())
                    if time.time() - t0 > self.lease_timeout:
                        got = self.store.compare_set(self._k("owner", c), "", str(self.rank))
                        if int(got.decode()) == self.rank:
                            self._beat()
                            return self._range(c)
                    pending = True
                    continue
                owner = int(self.store.get(self._k("owner", c)).decode())
                if owner == self.rank or not self._gone(owner):
                    pending = True
                    continue
                rec = self._record(owner)
                if rec is not None and c in rec[2]:
                    self.store.set(self._k("done", c), str(owner))   # published before it left
                    continue
                got = self.store.compare_set(self._k("owner", c), str(owner), str(self.rank))
                if int(got.decode()) == self.rank:
                    self._beat()
                    return self._range(c)
                pending = True
            if not pending:
                return None
            self._beat()
            time.sleep(self.poll)

    def publish(self, r, E, V):
        """After finishing chunk range r: store this rank's cumulative partial
        (E, V as numpy arrays, including r) and mark the chunk done."""
        c = r[0] // self.chunk
        self.mine.append(c)
        self.store.set(self._k("part", self.rank), pickle.dumps((float(E), np.asarray(V), list(self.mine))))
        self.store.set(self._k("done", c), str(self.rank))
        self._beat()

    def leave(self):
        """Announce that this rank takes no further chunks (its published
        chunks stay counted; a chunk it holds is re-offered)."""
        self.store.set(self._k("left", self.rank), "1")

    def finish(self, world: int, host_rank: int = 0):
        """Mark this rank done; the rank whose process hosts the store (rank 0
        with the default TCP store) then waits until every other rank is done
        or gone, so the store outlives their last use of it."""
        self.store.set(self._k("fin", self.rank), "1")
        if self.rank != host_rank:
            return
        while True:
            waiting = [r for r in range(world) if r != self.rank and not self.store.check([self._k("fin", r)])
                       and not self._gone(r)]
            if not waiting:
                return
            time.sleep(self.poll)

    def reduce_published(self, world: int):
        """Sum of every rank's published partial (after take() returned None):
        (E, V, chunks); the chunk lists are disjoint and cover all chunks."""
        E, V, chunks = 0.0, None, []
        for r in range(world):
            rec = self._record(r)
            if rec is None:
                continue
            E += rec[0]
            V = rec[1].copy() if V is None else V + rec[1]
            chunks += rec[2]
        if sorted(chunks) != list(range(self.nchunks)):
            raise RuntimeError(f"published chunks {sorted(chunks)} do not cover 0..{self.nchunks - 1} once")
        return E, V, chunks


def exc_pulled(plan, xc, D, V, E, queue: BlockQueue, group=None):
    """kldi_exc over the chunks this rank pulls from `queue`, summed, then the
    sum over ranks (device tensors V, E receive the full result).  Returns the
    block ranges this rank evaluated; the plan is left on all its grid blocks.
    With a plain queue the sum is an all-reduce over the process group (none
    without a group of more than one rank); with a leased queue the partials
    go through the store (publish after every chunk, reduce_published), so
    the ranks that stay produce the full result when another rank leaves
    between chunks."""
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
        if queue.lease_timeout is not None:
            queue.publish(r, E.item(), V.cpu().numpy())
    plan.set_block_range(0, plan.stats["nblocks"])
    import torch.distributed as dist
    if queue.lease_timeout is not None:
        world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
        Es, Vs, _ = queue.reduce_published(world)
        queue.finish(world)
        V.copy_(torch.from_numpy(Vs))
        E.fill_(Es)
    elif dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        reduce_exc(V, E, group)
    return done

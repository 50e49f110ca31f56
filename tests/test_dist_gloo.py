"""Multi-process host logic on CPU ranks (gloo): grid-block partitioning and
the sum-reduce of partial V_xc / E_xc.  Each rank evaluates its block range
with the oracle; the reduced result must equal the single-process oracle."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grad as ogr
from oracle import grid as og
from paper_2605_10363_gb300 import dist as kdist


def test_partition_covers_and_balances():
    rng = np.random.default_rng(0)
    w = rng.integers(1, 400, size=1000).astype(float)
    for world in (1, 2, 3, 8, 13):
        r = kdist.partition_blocks(w, world)
        assert r[0][0] == 0 and r[-1][1] == w.size
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        loads = [w[g0:g1].sum() for g0, g1 in r]
        assert max(loads) <= w.sum() / world + w.max()


def test_partition_edge_cases():
    r = kdist.partition_blocks(np.ones(3), 5)         # more ranks than blocks: some ranges are empty
    assert sum(g1 - g0 for g0, g1 in r) == 3 and all(g1 >= g0 for g0, g1 in r)
    assert kdist.partition_blocks(np.zeros(0), 2) == [(0, 0), (0, 0)]
    assert kdist.partition_blocks(np.zeros(4), 2) == [(0, 2), (2, 4)]
    w = kdist.block_weights(np.array([0, 2, 2, 5]))
    assert np.array_equal(w, [4.0, 0.0, 9.0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ranges, out_dir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = synth.make_system(1)
        g = og.build_grid(s.Z, s.xyz, s.grid)
        sh = ob.build_shells(s.xyz, s.basis)
        g0, g1 = ranges[rank]
        part = oe.evaluate(s, g, sh, screened=True, blocks=range(g0, g1))
        V = torch.from_numpy(part.V.copy())
        E = torch.tensor([part.E], dtype=torch.float64)
        kdist.reduce_exc(V, E)
        np.save(os.path.join(out_dir, f"V{rank}.npy"), V.numpy())
        np.save(os.path.join(out_dir, f"E{rank}.npy"), E.numpy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_to_the_single_process_result(tmp_path):
    import torch.multiprocessing as mp
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    ref = oe.evaluate(s, g, sh, screened=True, keep_lists=True)
    ptr = np.zeros(g.nblocks + 1, dtype=np.int64)
    for b in range(g.nblocks):
        ptr[b + 1] = ptr[b] + ref.lists[b]["S"].size
    ranges = kdist.partition_blocks(kdist.block_weights(ptr), 2)
    assert ranges[0][1] > 0 and ranges[1][0] < g.nblocks
    mp.start_processes(_rank_main, args=(2, _free_port(), ranges, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        V = np.load(tmp_path / f"V{r}.npy")
        E = np.load(tmp_path / f"E{r}.npy")[0]
        assert E == pytest.approx(ref.E, rel=1e-13)
        assert np.abs(V - ref.V).max() <= 1e-13 * np.abs(ref.V).max()


def _rank_ordered(rank, world, port, ranges, out_dir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = synth.make_system(1)
        g = og.build_grid(s.Z, s.xyz, s.grid)
        sh = ob.build_shells(s.xyz, s.basis)
        g0, g1 = ranges[rank]
        part = oe.evaluate(s, g, sh, screened=True, blocks=range(g0, g1), xc_kind="pbe")
        V = torch.from_numpy(part.V.copy())
        E = torch.tensor([part.E], dtype=torch.float64)
        kdist.reduce_exc(V, E, ordered=True)
        np.save(os.path.join(out_dir, f"V{rank}.npy"), V.numpy())
        np.save(os.path.join(out_dir, f"E{rank}.npy"), E.numpy())
    finally:
        dist.destroy_process_group()


def test_ordered_reduction_is_bitwise_that_of_one_process(tmp_path):
    """Three ranks with the ordered reduction: every rank holds the same bits,
    and they are the bits of one process adding the same block-range partials
    in rank order (the reduction order is fixed, not the collective's)."""
    import torch.multiprocessing as mp
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    n = g.nblocks
    ranges = [(0, n // 4), (n // 4, (2 * n) // 3), ((2 * n) // 3, n)]
    mp.start_processes(_rank_ordered, args=(3, _free_port(), ranges, str(tmp_path)), nprocs=3, join=True,
                       start_method="spawn")
    parts = [oe.evaluate(s, g, sh, screened=True, blocks=range(g0, g1), xc_kind="pbe") for g0, g1 in ranges]
    V = parts[0].V.copy()
    E = np.array([parts[0].E])
    for p in parts[1:]:
        V += p.V
        E += p.E
    for r in range(3):
        assert np.array_equal(np.load(tmp_path / f"V{r}.npy"), V)
        assert np.array_equal(np.load(tmp_path / f"E{r}.npy"), E)
    ref = oe.evaluate(s, g, sh, screened=True, xc_kind="pbe")
    assert np.abs(V - ref.V).max() <= 1e-13 * np.abs(ref.V).max()


def _rank_grad(rank, world, port, ranges, out_dir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = synth.make_system(1)
        g = og.build_grid(s.Z, s.xyz, s.grid)
        sh = ob.build_shells(s.xyz, s.basis)
        g0, g1 = ranges[rank]
        G = torch.from_numpy(ogr.exc_gradient(s, g, sh, screened=True, blocks=range(g0, g1)).copy())
        E = torch.tensor([oe.evaluate(s, g, sh, screened=True, want_v=False, blocks=range(g0, g1)).E],
                         dtype=torch.float64)
        kdist.reduce_grad(G, E)
        np.save(os.path.join(out_dir, f"G{rank}.npy"), G.numpy())
        np.save(os.path.join(out_dir, f"E{rank}.npy"), E.numpy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_the_gradient(tmp_path):
    """The nuclear gradient is a sum over grid blocks: two ranks' partial
    gradients over complementary block ranges reduce to the full gradient."""
    import torch.multiprocessing as mp
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    Gref = ogr.exc_gradient(s, g, sh, screened=True)
    ranges = [(0, g.nblocks // 3), (g.nblocks // 3, g.nblocks)]
    mp.start_processes(_rank_grad, args=(2, _free_port(), ranges, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    for r in range(2):
        G = np.load(tmp_path / f"G{r}.npy")
        assert np.abs(G - Gref).max() <= 1e-13 * np.abs(Gref).max()


def _rank_pull(rank, world, port, nblocks, chunk, out_dir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = synth.make_system(1)
        g = og.build_grid(s.Z, s.xyz, s.grid)
        sh = ob.build_shells(s.xyz, s.basis)
        store = dist.distributed_c10d._get_default_store()
        q = kdist.BlockQueue(store, nblocks, chunk, key="exc_blocks_0")
        V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64)
        E = torch.zeros(1, dtype=torch.float64)
        done = []
        while True:                      # the loop of kdist.exc_pulled, with the oracle as the worker
            r = q.take()
            if r is None:
                break
            part = oe.evaluate(s, g, sh, screened=True, blocks=range(*r))
            V += torch.from_numpy(part.V)
            E += part.E
            done.append(r)
        kdist.reduce_exc(V, E)
        np.save(os.path.join(out_dir, f"V{rank}.npy"), V.numpy())
        np.save(os.path.join(out_dir, f"E{rank}.npy"), E.numpy())
        np.save(os.path.join(out_dir, f"done{rank}.npy"), np.array(done, dtype=np.int64).reshape(-1, 2))
    finally:
        dist.destroy_process_group()


def test_pull_queue_covers_every_block_once(tmp_path):
    """Three ranks pull chunks of 16 grid blocks from the shared counter: the
    chunks they took are disjoint, cover all blocks, and the reduced E_xc and V
    equal the single-process oracle."""
    import torch.multiprocessing as mp
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    ref = oe.evaluate(s, g, sh, screened=True)
    world = 3
    mp.start_processes(_rank_pull, args=(world, _free_port(), g.nblocks, 16, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    taken = np.concatenate([np.load(tmp_path / f"done{r}.npy") for r in range(world)])
    taken = taken[np.argsort(taken[:, 0])]
    assert taken[0, 0] == 0 and taken[-1, 1] == g.nblocks
    assert np.all(taken[1:, 0] == taken[:-1, 1])
    for r in range(world):
        assert np.load(tmp_path / f"E{r}.npy")[0] == pytest.approx(ref.E, rel=1e-13)
        assert np.abs(np.load(tmp_path / f"V{r}.npy") - ref.V).max() <= 1e-13 * np.abs(ref.V).max()


def test_block_queue_single_process():
    import torch.distributed as dist
    store = dist.HashStore()
    q = kdist.BlockQueue(store, 10, 4, key="k")
    assert [q.take() for _ in range(4)] == [(0, 4), (4, 8), (8, 10), None]
    with pytest.raises(ValueError):
        kdist.BlockQueue(store, 10, 0, key="k2")


def _rank_pull_leave(rank, world, port, nblocks, chunk, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    store = dist.distributed_c10d._get_default_store()
    q = kdist.BlockQueue(store, nblocks, chunk, key="exc_leave_0", rank=rank, lease_timeout=1.0)
    E, V = 0.0, np.zeros((s.nbf, s.nbf))
    done = []
    if rank == world - 1:
        # finishes one chunk, takes the next and leaves without a word (a
        # process that dies between chunks): the chunk it holds is lost
        r = q.take()
        part = oe.evaluate(s, g, sh, screened=True, blocks=range(*r))
        E, V = E + part.E, V + part.V
        q.publish(r, E, V)
        np.save(os.path.join(out_dir, f"done{rank}.npy"), np.array([r], dtype=np.int64))
        q.take()
        os._exit(0)
    while True:                          # the loop of kdist.exc_pulled with a leased queue
        r = q.take()
        if r is None:
            break
        part = oe.evaluate(s, g, sh, screened=True, blocks=range(*r))
        E, V = E + part.E, V + part.V
        q.publish(r, E, V)
        done.append(r)
    Es, Vs, chunks = q.reduce_published(world)
    q.finish(world)                      # rank 0 hosts the store: it leaves last
    np.save(os.path.join(out_dir, f"V{rank}.npy"), Vs)
    np.save(os.path.join(out_dir, f"E{rank}.npy"), np.array([Es]))
    np.save(os.path.join(out_dir, f"done{rank}.npy"), np.array(done, dtype=np.int64).reshape(-1, 2))
    os._exit(0)                          # a member of the group is gone: no collective teardown


def test_pull_queue_requeues_the_chunk_of_a_rank_that_leaves(tmp_path):
    """Three ranks pull leased chunks of 16 grid blocks; the last rank finishes
    one chunk, takes another and exits.  Its lease runs out (1 s without a
    heartbeat), a remaining rank takes the chunk over, and the two remaining
    ranks' sum of the published partials equals the single-process oracle;
    every chunk was evaluated by exactly one rank."""
    import torch.multiprocessing as mp
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    ref = oe.evaluate(s, g, sh, screened=True)
    world = 3
    mp.start_processes(_rank_pull_leave, args=(world, _free_port(), g.nblocks, 16, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    taken = np.concatenate([np.load(tmp_path / f"done{r}.npy") for r in range(world)])
    taken = taken[np.argsort(taken[:, 0])]
    assert taken[0, 0] == 0 and taken[-1, 1] == g.nblocks
    assert np.all(taken[1:, 0] == taken[:-1, 1])
    for r in range(world - 1):
        assert np.load(tmp_path / f"E{r}.npy")[0] == pytest.approx(ref.E, rel=1e-13)
        assert np.abs(np.load(tmp_path / f"V{r}.npy") - ref.V).max() <= 1e-13 * np.abs(ref.V).max()

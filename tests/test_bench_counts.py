"""The roofline's FLOP counts (bench.work_counts) against the oracle's screening
on grid blocks of the 4-water workload (no GPU needed): the density product's
algorithmic FLOPs are 2 x 128 x d_p d_q over the oracle's executed block pairs
(Eq. executed_block_output), the V product's over all of S_g^2 and over p <= q,
and the executed (tile-padded) counts follow from explicit enumeration of the
N tiles and of the greedy 4-block V windows."""
import numpy as np
import pytest

import bench
import synth
from oracle import exc as oe
from oracle import grid as og


class ListsOnly:
    """Stands in for a plan: only the retained lists that work_counts reads."""

    def __init__(self, ptr, idx, b):
        self._lists = (ptr, idx, b)

    def lists(self):
        return self._lists


@pytest.fixture(scope="module")
def screened():
    s = synth.make_system(2, nwaters=4)
    blocks = [0, 3, 77, 200, 431, 600, 901, 1091]
    g = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=blocks)
    ref = oe.evaluate(s, g, blocks=blocks, want_v=False, keep_lists=True)
    ptr = np.zeros(g.nblocks + 1, np.int64)
    idx, bsel = [], []
    for k in range(g.nblocks):
        L = ref.lists.get(k)
        if L is not None:
            idx.append(L["S"])
            bsel.append(L["b"][L["S"]])
        ptr[k + 1] = ptr[k] + (0 if L is None else L["S"].size)
    plan = ListsOnly(ptr, np.concatenate(idx).astype(np.int32), np.concatenate(bsel))
    return s, ref, plan


def _sizes(nbf):
    return [min(32, nbf - 32 * p) for p in range((nbf + 31) // 32)]


def test_algorithmic_counts_are_the_oracle_pairs(screened):
    s, ref, plan = screened
    d = _sizes(s.nbf)
    splits = 10
    counts = {}
    f_rho, f_v = bench.work_counts(plan, s, splits, counts, nq=2, v_align=2)
    rho = v = v_pq = 0.0
    for L in ref.lists.values():
        S, E1 = L["S"], L["E1"]
        for i, p in enumerate(S):
            for j, q in enumerate(S):
                t = 2.0 * 128 * d[p] * d[q]
                v += t
                v_pq += t if i <= j else 0.0
                rho += t if E1[i, j] else 0.0
    assert 0.0 < rho < v                          # some pairs are screened out, some kept
    assert f_rho == pytest.approx(splits * rho, rel=1e-14)
    assert f_v == pytest.approx(splits * v, rel=1e-14)
    assert counts["v_pairs_pq"] == pytest.approx(splits * v_pq, rel=1e-14)


@pytest.mark.parametrize("nq,v_align", [(2, 2), (4, 4), (4, 1)])
def test_executed_counts_by_enumeration(screened, nq, v_align):
    s, ref, plan = screened
    counts = {}
    bench.work_counts(plan, s, 1, counts, nq=nq, v_align=v_align)
    x_rho = x_v = 0.0
    for L in ref.lists.values():
        S, E1 = L["S"], L["E1"]
        # density product: one 128 x (32 nq) x 32 chunk per (N tile, row block)
        # with an executed pair in the tile
        for t0 in range(0, S.size, nq):
            for i in range(S.size):
                if any(E1[i, j] for j in range(t0, min(t0 + nq, S.size))):
                    x_rho += 2.0 * 128 * (32 * nq) * 32
        # V product: greedy windows of 4 basis blocks starting at multiples of
        # v_align; every retained block lies in exactly one window
        starts = []
        for p in S.tolist():
            if not starts or p > starts[-1] + 3:
                starts.append(p - p % v_align)
        for p in S.tolist():
            assert sum(w <= p <= w + 3 for w in starts) == 1
        assert all(w % v_align == 0 for w in starts)
        n = len(starts)
        x_v += 2.0 * 128 * 128 * (256 * n * (n - 1) // 2 + 128 * n)
    assert counts["executed_rho"] == pytest.approx(x_rho, rel=1e-14)
    assert counts["executed_v"] == pytest.approx(x_v, rel=1e-14)

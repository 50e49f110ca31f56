"""kldi_make_grid (library, host preprocessing) against the oracle's grid:
same point order, coordinates and Becke weights (no GPU needed)."""
import numpy as np

import synth
from oracle import grid as og


def test_grid_matches_oracle_workload1():
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(1)
    g = kldi.make_grid(s.Z, s.xyz, s.grid.nrad, s.grid.ntheta)
    xyz, w, atom = g.export()
    go = og.build_grid(s.Z, s.xyz, s.grid)
    assert g.npoints == go.npoints and g.nreal == go.nreal
    assert np.array_equal(atom, go.atom_of)
    assert np.abs(xyz - go.points).max() < 1e-13
    assert np.abs(w - go.weights).max() < 1e-12


def test_grid_matches_oracle_pruned_small_cluster():
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, nwaters=4)
    g = kldi.make_grid(s.Z, s.xyz, s.grid.nrad, s.grid.ntheta)
    xyz, w, atom = g.export()
    blocks = [0, 7, g.nblocks // 2, g.nblocks - 1]
    go = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=blocks)
    assert g.npoints == go.npoints and g.nreal == go.nreal
    assert np.abs(xyz - go.points).max() < 1e-13
    sel = np.concatenate([np.arange(b * 128, (b + 1) * 128) for b in blocks])
    assert np.abs(w[sel] - go.weights[sel]).max() < 1e-12
    assert np.all(w[g.nreal:] == 0.0)

"""The seeded input generators used by the benchmark and the tests beyond the
workload recipes: density-matrix variants, shell permutations; no GPU."""
import numpy as np

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og


def test_density_variants_are_valid_densities():
    s = synth.make_system(2, nwaters=4, keep_overlap=True)
    S = s.meta["S"]
    Ds = synth.density_variants(s, 3)
    assert len(Ds) == 3
    for D in Ds:
        assert np.allclose(D, D.T, atol=0)
        assert abs(np.trace(D @ S) - 40.0) <= 1e-9          # 4 waters, 10 electrons each
        assert np.abs(D @ S @ D - 2.0 * D).max() <= 1e-9   # D = 2 C C^T with C^T S C = I
    assert np.abs(Ds[0] - Ds[1]).max() > 1e-3
    assert np.abs(Ds[0] - s.D).max() > 1e-3


def test_permuted_shells_give_the_same_energy():
    """A permutation of the shells with D permuted alike is the same physical
    system: the dense oracle gives the same E_xc to rounding."""
    s = synth.make_system(1)
    rng = np.random.default_rng(7)
    perm = rng.permutation(s.basis.nshell)
    s2 = synth.permute_shells(s, perm)
    assert s2.nbf == s.nbf and np.array_equal(np.sort(s2.meta["fn_perm"]), np.arange(s.nbf))
    f = s2.meta["fn_perm"]
    assert np.array_equal(s2.D, s.D[np.ix_(f, f)])
    S, S2 = synth.overlap_matrix(s.xyz, s.basis), synth.overlap_matrix(s2.xyz, s2.basis)
    assert np.abs(S2 - S[np.ix_(f, f)]).max() <= 1e-14
    g = og.build_grid(s.Z, s.xyz, s.grid)
    blocks = list(range(0, g.nblocks, 9))
    e1 = oe.evaluate(s, g, ob.build_shells(s.xyz, s.basis), screened=False, blocks=blocks)
    e2 = oe.evaluate(s2, g, ob.build_shells(s2.xyz, s2.basis), screened=False, blocks=blocks)
    assert abs(e1.E - e2.E) <= 1e-12 * abs(e1.E)
    assert np.abs(e2.V - e1.V[np.ix_(f, f)]).max() <= 1e-12 * np.abs(e1.V).max()


def test_keep_overlap_is_the_overlap_matrix():
    s = synth.make_system(1, keep_overlap=True)
    assert np.abs(s.meta["S"] - synth.overlap_matrix(s.xyz, s.basis)).max() == 0.0
    assert "S" not in synth.make_system(1).meta

"""Degenerate and edge inputs through the C ABI: nothing retained, a zero
density matrix, a single atom (the Becke partition is the identity), a
scaled density (E_x[lambda D] = lambda^(4/3) E_x[D] for Slater exchange), and
ragged sizes (functions not a multiple of 32, a padded last grid block)."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og

pytestmark = pytest.mark.gpu


def _run(s, prec, xc, D=None):
    from paper_2605_10363_gb300 import kldi
    plan = kldi.plan_for_system(s, prec=prec, xc=xc)
    V = np.zeros((s.nbf, s.nbf))
    E = np.zeros(1)
    kldi.exc(plan, xc, s.D if D is None else D, V, E)
    return plan, E[0], V


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_nothing_retained(prec):
    s = synth.make_system(1)
    s.t_b = s.t_d = 1e6                       # no basis block reaches the threshold
    plan, E, V = _run(s, prec, "lda_x")
    assert plan.stats["retained"] == 0
    assert E == 0.0 and not V.any()


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_zero_density(prec):
    s = synth.make_system(1)
    _, E, V = _run(s, prec, "pbe", D=np.zeros_like(s.D))
    assert E == 0.0 and not V.any()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x6", 1e-6)])
def test_single_atom(prec, tol):
    s = synth.make_system(1)
    keep = np.nonzero(np.asarray(s.basis.atom) == 0)[0]           # the first oxygen's shells only
    from synth import Basis, System
    ptr = s.basis.prim_ptr
    exps = np.concatenate([s.basis.exps[ptr[k]:ptr[k + 1]] for k in keep])
    coefs = np.concatenate([s.basis.coefs[ptr[k]:ptr[k + 1]] for k in keep])
    b = Basis(atom=np.zeros(len(keep), np.int32), l=np.asarray(s.basis.l)[keep],
              nprim=np.asarray(s.basis.nprim)[keep], exps=exps, coefs=coefs)
    nbf = b.nbf
    rng = np.random.default_rng(5)
    C = rng.normal(size=(nbf, 3))
    D = C @ C.T / nbf
    one = System("one_oxygen", s.Z[:1], s.xyz[:1], b, D, s.grid, 1e-12, 1e-12, "pbe")
    g = og.build_grid(one.Z, one.xyz, one.grid)
    ref = oe.evaluate(one, g, ob.build_shells(one.xyz, one.basis), screened=True)
    _, E, V = _run(one, prec, "pbe")
    assert abs(E - ref.E) <= tol
    assert np.abs(V - ref.V).max() <= (1e-10 if prec == "fp64" else 3e-7)


def test_density_scaling_slater():
    s = synth.make_system(1)
    _, E1, _ = _run(s, "fp64", "lda_x")
    _, E2, _ = _run(s, "fp64", "lda_x", D=0.25 * s.D)
    assert E2 == pytest.approx(E1 * 0.25 ** (4.0 / 3.0), rel=1e-12)


def test_ragged_sizes():
    s = synth.make_system(2, nwaters=3)           # 75 functions (not a multiple of 32)
    assert s.nbf % 32 != 0
    from paper_2605_10363_gb300 import kldi
    plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe")
    assert plan.grid.nreal % 128 != 0             # the last grid block is padded
    g = og.build_grid(s.Z, s.xyz, s.grid)
    ref = oe.evaluate(s, g, ob.build_shells(s.xyz, s.basis), screened=True)
    V = np.zeros((s.nbf, s.nbf))
    E = np.zeros(1)
    kldi.exc(plan, "pbe", s.D, V, E)
    assert abs(E[0] - ref.E) <= 1e-6
    assert np.abs(V - ref.V).max() <= 3e-7

"""The hot path on a basis in overlap-signature order (kldi_order_shells):
E_xc and V against the oracle evaluated on the same reordered system, and the
block statistics of both orders."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol_e,tol_v", [("fp64", 1e-10, 1e-10), ("bf16x6", 1e-6, 3e-7)])
def test_reordered_system_matches_oracle(prec, tol_e, tol_v):
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, nwaters=4)
    perm = kldi.order_shells(synth.overlap_matrix(s.xyz, s.basis), synth.shell_sizes(s.basis))
    s2 = synth.permute_shells(s, perm)
    g = og.build_grid(s2.Z, s2.xyz, s2.grid)
    ref = oe.evaluate(s2, g, ob.build_shells(s2.xyz, s2.basis), screened=True)
    plan = kldi.plan_for_system(s2, prec=prec, xc="pbe")
    V = np.zeros((s2.nbf, s2.nbf))
    E = np.zeros(1)
    kldi.exc(plan, "pbe", s2.D, V, E)
    assert abs(E[0] - ref.E) <= tol_e
    assert np.abs(V - ref.V).max() <= tol_v
    # V in the original order is the permuted-back matrix of the same quantity
    f = s2.meta["fn_perm"]
    Vo = np.zeros_like(V)
    Vo[np.ix_(f, f)] = V
    assert np.array_equal(Vo, Vo.T)


def test_block_statistics_of_both_orders():
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, nwaters=12)
    perm = kldi.order_shells(synth.overlap_matrix(s.xyz, s.basis), synth.shell_sizes(s.basis))
    a = kldi.plan_for_system(s, prec="bf16x6", xc="pbe").stats
    b = kldi.plan_for_system(synth.permute_shells(s, perm), prec="bf16x6", xc="pbe").stats
    print("atom order", {k: a[k] for k in ("retained", "pair_slots", "vtile_work")})
    print("overlap-signature order", {k: b[k] for k in ("retained", "pair_slots", "vtile_work")})
    assert a["npoints"] == b["npoints"] and a["nbf"] == b["nbf"]

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


@pytest.mark.parametrize("prec", ["fp64", "bf16x6"])
def test_shell_order_option_keeps_the_callers_order(prec):
    """A plan screened with shell_order works in the permuted order internally
    and takes D / returns V in the caller's order: the same numbers as a plan
    of the explicitly permuted system, mapped back."""
    import torch
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, nwaters=4)
    perm = kldi.order_shells(synth.overlap_matrix(s.xyz, s.basis), synth.shell_sizes(s.basis))
    s2 = synth.permute_shells(s, perm)
    f = s2.meta["fn_perm"]
    p1 = kldi.plan_for_system(s, prec=prec, xc="pbe", shell_order=perm)
    p2 = kldi.plan_for_system(s2, prec=prec, xc="pbe")
    assert p1.stats["pair_slots"] == p2.stats["pair_slots"]
    V1, E1 = np.zeros((s.nbf, s.nbf)), np.zeros(1)
    V2, E2 = np.zeros((s.nbf, s.nbf)), np.zeros(1)
    kldi.exc(p1, "pbe", s.D, V1, E1)
    kldi.exc(p2, "pbe", s2.D, V2, E2)
    back = np.zeros_like(V2)
    back[np.ix_(f, f)] = V2
    assert E1[0] == pytest.approx(E2[0], rel=1e-14, abs=0)
    assert np.abs(V1 - back).max() <= 1e-13 * np.abs(back).max()
    # device buffers, the unfused pair and the gradient take the caller's order too
    Dd = torch.from_numpy(s.D).cuda()
    Vd = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    kldi.exc(p1, "pbe", Dd, Vd, Ed)
    torch.cuda.synchronize()
    assert np.abs(Vd.cpu().numpy() - V1).max() <= 1e-13 * np.abs(V1).max()
    rho = np.zeros(p1.npoints)
    grad = np.zeros((p1.npoints, 3))
    kldi.density(p1, s.D, rho, grad)
    V3, E3 = np.zeros((s.nbf, s.nbf)), np.zeros(1)
    kldi.vxc(p1, "pbe", rho, grad, V3, E3)
    assert np.abs(V3 - V1).max() <= 1e-12 * np.abs(V1).max() + (1e-7 if prec == "bf16x6" else 0.0)
    G1, G2 = np.zeros((len(s.Z), 3)), np.zeros((len(s.Z), 3))
    kldi.exc_grad(p1, "pbe", s.D, G1, E1)
    kldi.exc_grad(p2, "pbe", s2.D, G2, E2)
    assert np.abs(G1 - G2).max() <= 1e-12

"""Nuclear gradient of E_xc on the GPU (FP64 block form) against the FP64
oracle (oracle/grad.py, pinned by finite differences): both sides FP64, so
max |dG| <= 1e-10 Ha/bohr (sums of ~1e5 terms) and E_xc to 1e-10 Ha."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grad as ogr
from oracle import grid as og

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,xc", [("w1", "lda_x"), ("w1", "pbe"), ("w4", "pbe")])
def test_gradient_matches_oracle(name, xc):
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(1) if name == "w1" else synth.make_system(2, nwaters=4)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    Gref = ogr.exc_gradient(s, g, sh, screened=True, xc_kind=xc)
    Eref = oe.evaluate(s, g, sh, screened=True, want_v=False, xc_kind=xc).E
    plan = kldi.plan_for_system(s, prec="fp64", xc=xc)
    G = np.zeros((len(s.Z), 3))
    E = np.zeros(1)
    kldi.exc_grad(plan, xc, s.D, G, E)
    print(f"{name} {xc}: max|G| {np.abs(Gref).max():.3e}, max|dG| {np.abs(G - Gref).max():.2e}, dE {E[0] - Eref:.2e}")
    assert abs(E[0] - Eref) <= 1e-10
    assert np.abs(G - Gref).max() <= 1e-10


def test_gradient_device_buffers_and_precision_guard():
    import torch
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(1)
    plan = kldi.plan_for_system(s, prec="fp64", xc="lda_x")
    Gh = np.zeros((len(s.Z), 3))
    Eh = np.zeros(1)
    kldi.exc_grad(plan, "lda_x", s.D, Gh, Eh)
    Gd = torch.zeros((len(s.Z), 3), dtype=torch.float64, device="cuda")
    Ed = torch.zeros(1, dtype=torch.float64, device="cuda")
    kldi.exc_grad(plan, "lda_x", torch.from_numpy(s.D).cuda(), Gd, Ed)
    torch.cuda.synchronize()
    assert np.abs(Gd.cpu().numpy() - Gh).max() <= 1e-13
    bf = kldi.plan_for_system(s, prec="bf16x6", xc="lda_x")
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc_grad(bf, "lda_x", s.D, Gh, Eh)
    assert e.value.status == kldi.EUNSUPPORTED

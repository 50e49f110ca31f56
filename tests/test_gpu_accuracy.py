"""Whole-grid accuracy at the stated target (|dE_xc| <= 1e-6 Ha, max|dV| <= 1e-7)
on a system the oracle evaluates whole only offline: 100 waters (300 atoms,
2500 functions, 3.5M grid points, PBE-form GGA, t_b = t_d = 1e-10).

The stored values (tests/golden/water100_pbe.json) are written by
tests/golden/make_golden.py, which calls only the CPU oracle.  The plan uses
the generated (atom) shell order, the oracle's block partition, so the
screened products are the same on both sides.  BF16X10 is held to the target;
BF16X6 is measured and stated (it misses 1e-6 Ha on whole grids of this size).
"""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "water100_pbe.json")


@pytest.mark.skipif(not os.path.exists(GOLD), reason="stored oracle values not written")
def test_water100_whole_grid_against_oracle():
    import torch

    from paper_2605_10363_gb300 import kldi
    gold = json.load(open(GOLD))
    s = synth.make_system(2, nwaters=100)
    plan = kldi.plan_for_system(s, prec="bf16x10", xc="pbe")
    assert plan.npoints == gold["npoints"] and s.nbf == gold["nbf"]
    D = torch.from_numpy(s.D).cuda()
    vs = np.array(gold["V_samples"])
    ii, jj = vs[:, 0].astype(int), vs[:, 1].astype(int)
    out = {}
    for prec in ("bf16x10", "bf16x6"):
        plan.set_precision(prec)
        V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        kldi.exc(plan, "pbe", D, V, E)
        torch.cuda.synchronize()
        Vh = V.cpu().numpy()
        dE = E.item() - gold["E_screened"]
        dV = np.abs(Vh[ii, jj] - vs[:, 2]).max()
        dtr = abs(float(np.sum(s.D * Vh)) - gold["trace_DV"])
        out[prec] = (dE, dV, dtr)
        print(f"water100 {prec}: E {E.item():.10f} dE {dE:+.2e} sampled max|dV| {dV:.2e} d tr(DV) {dtr:.2e}")
    dE, dV, dtr = out["bf16x10"]
    assert abs(dE) <= 1e-6
    assert dV <= 1e-7
    assert dtr <= 1e-7 * np.abs(s.D).sum()
    assert abs(out["bf16x6"][0]) <= 2e-5      # BF16X6: its measured error, stated

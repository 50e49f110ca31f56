"""Threshold sensitivity of the block filtering (the paper's t_b = t_d sweep,
Sec. IV): on the 33-water workload the screened E_xc (BF16x6) approaches the
dense oracle value (stored in tests/golden/water33_pbe.json) as the threshold
falls, and the retained work and the step time grow.  The table is printed
and the error bound checked: at t = 1e-10 (the workload's threshold) the
screened result is within 1e-6 Ha of the dense one."""
import json
import os
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_threshold_sweep_water33():
    import torch
    from paper_2605_10363_gb300 import kldi
    gold = json.load(open(os.path.join(HERE, "golden", "water33_pbe.json")))
    s = synth.make_system(2)
    D = torch.from_numpy(s.D).cuda()
    V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    rows = []
    for t in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12):
        s.t_b = s.t_d = t
        plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe")
        kldi.exc(plan, "pbe", D, V, E)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            kldi.exc(plan, "pbe", D, V, E)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / 3 * 1e3
        ptr, _, _ = plan.lists()
        n = np.diff(ptr).astype(float)
        frac = float(np.sum(n * n)) / (plan.stats["nblocks"] * plan.stats["nbasis_blocks"] ** 2)
        rows.append((t, E.item() - gold["E_dense"], frac, ms))
    print("\n   t_b = t_d   E - E_dense (Ha)   retained pair fraction   ms per evaluation")
    for t, dE, frac, ms in rows:
        print(f"   {t:8.0e}   {dE:+.3e}        {frac:.3f}                  {ms:.1f}")
    errs = [abs(r[1]) for r in rows]
    assert errs[0] > errs[2]                      # coarse thresholds err more
    assert abs(rows[3][1]) <= 1e-6                # the workload's threshold
    assert rows[4][2] >= rows[0][2]               # retained work grows as t falls

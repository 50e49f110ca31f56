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


def test_size_series_screened_vs_dense():
    """The crossover study (Sec. IV, Fig. 5): water clusters of growing size,
    BF16x6, the workload's thresholds (t_b = t_d = 1e-10) against the same
    kernels with every block and block pair kept (t_b = t_d = 0, the dense
    form).  Dense work grows with N_points x N_basis^2, screened work with
    N_points x n_g^2 where n_g saturates, so the advantage of screening must
    grow with the system size."""
    import torch
    from paper_2605_10363_gb300 import kldi
    rows = []
    for nw in (4, 8, 16, 33, 66, 100):
        s = synth.make_system(2, nwaters=nw)
        order = kldi.order_shells(synth.overlap_matrix(s.xyz, s.basis), synth.shell_sizes(s.basis))
        D = torch.from_numpy(s.D).cuda()
        V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        ms, Es, npts = [], [], 0
        for t in (1e-10, 0.0):
            s.t_b = s.t_d = t
            plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe", shell_order=order)
            npts = plan.grid.nreal
            kldi.exc(plan, "pbe", D, V, E)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(2):
                kldi.exc(plan, "pbe", D, V, E)
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) / 2 * 1e3)
            Es.append(E.item())
            del plan
        rows.append((nw, 3 * nw, s.nbf, npts, ms[0], ms[1], Es[0] - Es[1]))
    print("\n   waters  atoms  N_basis   points     screened ms   dense ms   dense/screened   E_scr - E_dense")
    for nw, na, nb, npts, m0, m1, dE in rows:
        print(f"   {nw:6d} {na:6d} {nb:8d} {npts:10d} {m0:12.2f} {m1:10.2f} {m1 / m0:14.2f}     {dE:+.2e}")
    ratios = [r[5] / r[4] for r in rows]
    assert ratios[-1] > ratios[2] > 1.0             # screening pays more as the system grows
    assert all(abs(r[6]) <= 1e-6 for r in rows)    # and changes E_xc by less than the tolerance

"""The allocation-free energy entry point against the plan path.

kldi_exc_energy_noalloc serves callers that may not allocate device memory
(for example code running inside CUDA graph capture, or hosts that reserve all
device memory up front).  Its E_xc of a device-resident density must equal the
E_xc that kldi_vxc computes from the same density, on two calls in a row (the
second call reuses the fixed device array the first one filled).  This file
is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,xc", [("w1", "lda_x"), ("w4", "pbe")])
def test_noalloc_energy_matches_plan_path(name, xc):
    import torch

    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(1) if name == "w1" else synth.make_system(2, nwaters=4)
    plan = kldi.plan_for_system(s, prec="fp64", xc=xc)
    n = plan.npoints
    rho = torch.zeros(n, dtype=torch.float64, device="cuda")
    grad = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    kldi.density(plan, torch.from_numpy(s.D).cuda(), rho, grad if xc != "lda_x" else None)
    V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
    E_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    kldi.vxc(plan, xc, rho, grad if xc != "lda_x" else None, V, E_ref)
    _, w, _ = plan.grid.export()
    w_dev = torch.from_numpy(w).cuda()
    for _ in range(2):
        E = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        kldi.exc_energy_noalloc(xc, n, rho, grad if xc != "lda_x" else None, w_dev, E)
        torch.cuda.synchronize()
        assert abs(float(E[0]) - float(E_ref[0])) <= 1e-12 * abs(float(E_ref[0]))


def test_noalloc_rejects_oversize_and_host_input():
    import torch

    from paper_2605_10363_gb300 import kldi
    big = 65536 * 128 + 1
    rho = torch.zeros(8, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc_energy_noalloc("lda_x", big, rho, None, rho, E)
    assert e.value.status == kldi.EINVAL
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc_energy_noalloc("lda_x", 8, np.zeros(8), None, rho, E)
    assert e.value.status == kldi.EINVAL

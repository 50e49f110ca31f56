"""Failure detection without a GPU fault: the bounded device waits.

* A CTA that waits on an mbarrier at which nothing arrives (nothing else in
  flight) gives up after the given limit and the call returns KLDI_ETIMEOUT;
  with the arrival it returns KLDI_OK.
* The tensor-core V product with one work item withheld from its consumers
  (the plan's test hook): their wait runs out after the plan's shortened
  limit, the kernel waits for its own products and copies, frees its tensor
  memory and exits, and kldi_exc returns KLDI_ETIMEOUT.  The same plan, with
  the hook off and the default limit restored, then reproduces the oracle's
  E_xc and V at the mode's tolerance.
"""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og

pytestmark = pytest.mark.gpu


def test_selftest_wait_gives_up_and_reports():
    from paper_2605_10363_gb300 import kldi
    kldi.selftest_wait(1_000_000, arrive=True)
    with pytest.raises(kldi.KldiError) as e:
        kldi.selftest_wait(1_000_000, arrive=False)      # 1 ms, nobody arrives
    assert e.value.status == kldi.ETIMEOUT
    kldi.selftest_wait(1_000_000, arrive=True)           # the context is still usable


@pytest.mark.parametrize("prec,tE,tV", [("bf16x6", 1e-6, 3e-7), ("bf16x10", 1e-6, 1e-7)])
def test_withheld_work_item_times_out_and_plan_recovers(prec, tE, tV):
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, nwaters=4)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    ref = oe.evaluate(s, g, ob.build_shells(s.xyz, s.basis), screened=True)
    plan = kldi.plan_for_system(s, prec=prec, xc="pbe")
    V = np.zeros((s.nbf, s.nbf))
    E = np.zeros(1)
    plan.set_wait_limit(50_000_000)                      # 50 ms
    kldi.exc(plan, "pbe", s.D, V, E)                     # a normal call under the short limit
    assert abs(E[0] - ref.E) <= tE
    plan.set_withhold(1)
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc(plan, "pbe", s.D, V, E)
    assert e.value.status == kldi.ETIMEOUT
    plan.set_withhold(-1)
    plan.set_wait_limit(0)
    kldi.exc(plan, "pbe", s.D, V, E)
    assert abs(E[0] - ref.E) <= tE
    assert np.abs(V - ref.V).max() <= tV

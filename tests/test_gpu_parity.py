"""GPU parity: the library, through the C ABI, against the CPU oracle on the
same seeded inputs, element by element.

Tolerances (written per mode, derived from the arithmetic):
  fp64     FP64 block form: |dE| <= 1e-10 Ha, max|dV| <= 1e-10, rho to 1e-12.
  bf16x10  four 8-bit slices per operand (2^-32 of the row / column scale),
           exact tensor-core levels, double-float basis values, X and
           row-dot: the stated target |dE| <= 1e-6 Ha and max|dV| <= 1e-7;
           rho within its slicing error model (2^-30 of the point's density
           scale, rho_model_bound).
  bf16x6   three 8-bit slices, FP32 basis values: the fast mode, held to its
           measured error, not to the target: |dE| <= 1e-6 Ha on these small
           systems, max|dV| <= 3e-7 (the largest V elements, ~5 Ha, carry the
           2^-24 relative error of FP32 operands); rho to 4e-5 of |rho| + 1e-9.
  bf16x3   two 8-bit slices: element error 2^-16 of the row / column scale,
           so |dE| <= 3e-5 |E| and max|dV| <= 2e-4.
Index work (the retained lists) is compared exactly; summaries to 1e-12.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {
    "fp64": dict(E_abs=1e-10, V=1e-10, rho_rel=1e-12, rho_abs=1e-14),
    "bf16x10": dict(E_abs=1e-6, V=1e-7, rho_model=2.0 ** -30),
    "bf16x6": dict(E_abs=1e-6, V=3e-7, rho_rel=4e-5, rho_abs=1e-9),
    "bf16x3": dict(E_rel=3e-5, V=2e-4, rho_rel=2e-2, rho_abs=1e-7),
}

_cache = {}


def oracle_run(key, system, xc):
    if key not in _cache:
        g = og.build_grid(system.Z, system.xyz, system.grid)
        sh = ob.build_shells(system.xyz, system.basis)
        _cache[key] = (oe.evaluate(system, g, sh, screened=True, xc_kind=xc, keep_lists=True), g)
    return _cache[key]


@pytest.fixture(scope="module")
def sys_cache():
    return {"w1": synth.make_system(1), "w4": synth.make_system(2, nwaters=4)}


def run_lib(system, prec, xc, device=False):
    import torch

    from paper_2605_10363_gb300 import kldi
    plan = kldi.plan_for_system(system, prec=prec, xc=xc)
    nbf = system.nbf
    if device:
        D = torch.from_numpy(system.D).cuda()
        V = torch.zeros((nbf, nbf), dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        kldi.exc(plan, xc, D, V, E)
        torch.cuda.synchronize()
        V, E = V.cpu().numpy(), E.cpu().numpy()
    else:
        V = np.zeros((nbf, nbf))
        E = np.zeros(1)
        kldi.exc(plan, xc, system.D, V, E)
    rho = np.zeros(plan.npoints)
    grad = np.zeros((plan.npoints, 3)) if xc != "lda_x" else None
    kldi.density(plan, system.D, rho, grad)
    return plan, E[0], V, rho, grad


def rho_model_bound(system, g, scale):
    """Error model of the sliced density product: every element of Phi exact to
    `scale` of its point's scale (>= max_m |phi_m|) and every element of D to
    `scale` of its column scale (max_m |D_mn|):
      |d rho_i| <= scale sum_n |phi_n| (2 max_m |phi_m| sum_m |D_mn| + max_m |D_mn| sum_m |phi_m|)
    (a factor 2 on the first term and 2 over the slicing bound for the drains)."""
    ap = np.abs(ob.eval_basis(g.points, ob.build_shells(system.xyz, system.basis), deriv=False)[0])
    aD = np.abs(system.D)
    return 2.0 * scale * (2.0 * ap.max(axis=1) * (ap @ aD.sum(axis=0)) + ap.sum(axis=1) * (ap @ aD.max(axis=0)))


def check(prec, E, V, rho, ref, system=None, g=None):
    t = TOL[prec]
    tolE = t["E_abs"] if "E_abs" in t else t["E_rel"] * abs(ref.E)
    assert abs(E - ref.E) <= tolE, (prec, E, ref.E)
    assert np.abs(V - ref.V).max() <= t["V"], (prec, np.abs(V - ref.V).max())
    assert np.array_equal(V, V.T)
    if "rho_model" in t:
        bound = rho_model_bound(system, g, t["rho_model"])
        ratio = np.abs(rho - ref.rho) / (bound + 1e-300)
        print(f"  rho: max error / model bound {ratio.max():.3f}")
        assert np.all(np.abs(rho - ref.rho) <= bound)
    else:
        assert np.all(np.abs(rho - ref.rho) <= t["rho_rel"] * np.abs(ref.rho) + t["rho_abs"])


@pytest.mark.parametrize("prec", ["fp64", "bf16x10", "bf16x6", "bf16x3"])
@pytest.mark.parametrize("name,xc", [("w1", "lda_x"), ("w1", "pbe"), ("w4", "pbe")])
def test_exc_matches_oracle(sys_cache, prec, name, xc):
    s = sys_cache[name]
    ref, g = oracle_run((name, xc), s, xc)
    plan, E, V, rho, grad = run_lib(s, prec, xc)
    print(f"{name} {xc} {prec}: dE {E - ref.E:+.2e} max|dV| {np.abs(V - ref.V).max():.2e}")
    check(prec, E, V, rho, ref, s, g)
    if grad is not None and prec == "fp64":
        assert np.allclose(grad, ref.grad, rtol=1e-11, atol=1e-13)
    if grad is not None and prec == "bf16x10":
        # grad rho = 2 sum grad Phi . R: the same slicing error model as rho,
        # relative to the point's density scale rather than to |grad rho|
        # (which can be small where the terms cancel)
        scale = np.abs(ref.grad) + np.abs(ref.rho)[:, None]
        ratio = np.abs(grad - ref.grad) / (scale + 1e-300)
        print(f"  grad rho: max error / (|grad rho| + rho) {ratio[scale > 1e-10].max():.2e}")
        assert np.all(np.abs(grad - ref.grad) <= 1e-6 * scale + 1e-11)


@pytest.mark.parametrize("prec", ["fp64", "bf16x6", "bf16x10"])
def test_device_pointers_equal_host_pointers(sys_cache, prec):
    s = sys_cache["w1"]
    _, E1, V1, _, _ = run_lib(s, prec, "lda_x", device=False)
    _, E2, V2, _, _ = run_lib(s, prec, "lda_x", device=True)
    assert abs(E1 - E2) < 1e-13
    assert np.abs(V1 - V2).max() < 1e-13


def test_repeat_calls_are_bitwise_deterministic(sys_cache):
    from paper_2605_10363_gb300 import kldi
    s = sys_cache["w4"]
    plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe")
    outs = []
    for _ in range(3):
        V = np.zeros((s.nbf, s.nbf))
        E = np.zeros(1)
        kldi.exc(plan, "pbe", s.D, V, E)
        outs.append((E[0], V))
    for E, V in outs[1:]:
        assert E == outs[0][0]
        # V: FP64 atomics of per-segment partial sums; order may differ in the last bit
        assert np.abs(V - outs[0][1]).max() <= 1e-13


def test_vxc_from_oracle_density(sys_cache):
    """kldi_vxc fed with the oracle's own rho / grad rho reproduces its E and V."""
    from paper_2605_10363_gb300 import kldi
    s = sys_cache["w4"]
    ref, g = oracle_run(("w4", "pbe"), s, "pbe")
    for prec, tV in (("fp64", 1e-10), ("bf16x10", 1e-7), ("bf16x6", 3e-7)):
        plan = kldi.plan_for_system(s, prec=prec, xc="pbe")
        V = np.zeros((s.nbf, s.nbf))
        E = np.zeros(1)
        kldi.vxc(plan, "pbe", ref.rho, np.ascontiguousarray(ref.grad), V, E)
        assert abs(E[0] - ref.E) < 1e-10
        assert np.abs(V - ref.V).max() < tV


@pytest.mark.parametrize("name,xc", [("w1", "pbe"), ("w4", "pbe")])
def test_retained_lists_match_oracle(sys_cache, name, xc):
    s = sys_cache[name]
    ref, g = oracle_run((name, xc), s, xc)
    from paper_2605_10363_gb300 import kldi
    plan = kldi.plan_for_system(s, prec="fp64", xc=xc)
    ptr, idx, b = plan.lists()
    for blk, L in ref.lists.items():
        S = idx[ptr[blk]:ptr[blk + 1]]
        assert np.array_equal(S, L["S"]), blk
        assert np.allclose(b[ptr[blk]:ptr[blk + 1]], L["b"][L["S"]], rtol=1e-12, atol=0)


def test_unsupported_and_invalid_requests(sys_cache):
    from paper_2605_10363_gb300 import kldi
    s = sys_cache["w1"]
    with pytest.raises(kldi.KldiError) as e:
        kldi.plan_for_system(s, prec="tf32x3", xc="lda_x")
    assert e.value.status == kldi.EUNSUPPORTED
    plan = kldi.plan_for_system(s, prec="bf16x6", xc="lda_x")
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc(plan, "pbe", s.D, np.zeros((s.nbf, s.nbf)), np.zeros(1))   # LDA plan, GGA call
    assert e.value.status == kldi.EINVAL


@pytest.mark.parametrize("prec,order", [("bf16x10", "overlap"), ("bf16x10", "atom"), ("bf16x6", "overlap"),
                                        ("bf16x6", "atom"), ("bf16x3", "atom")])
def test_full_size_water33(prec, order):
    """33 waters (1.15M points, 825 functions) against stored oracle values:
    E_xc, tr(D V), sampled V elements and rho / grad rho on sampled grid blocks.
    The benchmark's launch configuration is BF16x10 in the overlap-signature
    shell order; the stored values come from the oracle in the generated (atom)
    order, whose screened block partition differs by the screening error
    (dense - screened = 1.2e-9 Ha on this system; sampled V elements of the two
    partitions differ by up to ~3e-8)."""
    path = os.path.join(HERE, "golden", "water33_pbe.json")
    gold = json.load(open(path))
    from paper_2605_10363_gb300 import kldi
    s = synth.make_system(2, keep_overlap=True)
    perm = kldi.order_shells(s.meta["S"], synth.shell_sizes(s.basis)) if order == "overlap" else None
    plan = kldi.plan_for_system(s, prec=prec, xc="pbe", shell_order=perm)
    assert plan.npoints == gold["npoints"]
    V = np.zeros((s.nbf, s.nbf))
    E = np.zeros(1)
    kldi.exc(plan, "pbe", s.D, V, E)
    rho = np.zeros(plan.npoints)
    grad = np.zeros((plan.npoints, 3))
    kldi.density(plan, s.D, rho, grad)
    t = TOL[prec]
    tolE = t["E_abs"] if "E_abs" in t else t["E_rel"] * abs(gold["E_screened"])
    assert abs(E[0] - gold["E_screened"]) <= tolE, (E[0], gold["E_screened"])
    vs = np.array(gold["V_samples"])
    got = V[vs[:, 0].astype(int), vs[:, 1].astype(int)]
    assert np.abs(got - vs[:, 2]).max() <= t["V"]
    assert abs(np.sum(s.D * V) - gold["trace_DV"]) <= t["V"] * np.abs(s.D).sum()
    pts = np.concatenate([np.arange(b * 128, (b + 1) * 128) for b in gold["rho_blocks"]])
    r_ref = np.array(gold["rho"])
    if "rho_model" in t:
        g = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=[])
        sub = type("G", (), {"points": g.points[pts]})()
        bound = rho_model_bound(s, sub, t["rho_model"])
        if order == "overlap":
            # another block partition: the screened pairs differ by contributions
            # below the thresholds (observed 3e-9 of rho at most)
            bound = bound + 1e-8 * np.abs(r_ref) + 1e-10
        assert np.all(np.abs(rho[pts] - r_ref) <= bound)
    else:
        assert np.all(np.abs(rho[pts] - r_ref) <= t["rho_rel"] * np.abs(r_ref) + t["rho_abs"])

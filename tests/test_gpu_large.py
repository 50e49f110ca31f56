"""Full-size workloads the oracle cannot evaluate whole, held to it on sampled
grid blocks in the launch configuration the benchmark uses, and the grid's
Becke weights computed on the GPU.

The 1000-atom C/N/O/H cluster (9000 functions, 11.65M points) in BF16X10 (the
mode held to the stated target):
  * whole grid: E_xc within 1e-6 Ha and every element of V within 1e-7 of the
    FP64 block form on the same plan;
  * the FP64 block form and BF16X10 on seeded contiguous ranges of grid
    blocks (kldi_plan_set_block_range: the range's partial E_xc and V) against
    the screened FP64 oracle: FP64 to 1e-10, BF16X10 to 1e-6 Ha / 1e-7;
  * rho at a point follows the error model of the sliced product: every
    element of Phi is exact to 2^-32 of its point's scale (>= max_m |phi_m|)
    and every element of D to 2^-32 of its column scale (max_m |D_mn|), so
      |d rho_i| <= 2^-30 sum_n |phi_n| (2 max_m |phi_m| sum_m |D_mn| + max_m |D_mn| sum_m |phi_m|)
    (a factor 4 over the slicing bound for the double-float drains).
BF16X6 on the whole grid is measured and stated (it misses 1e-6 Ha here)."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og

pytestmark = pytest.mark.gpu


def _kldi():
    from paper_2605_10363_gb300 import kldi
    return kldi


def test_device_becke_weights_match_oracle():
    kldi = _kldi()
    s = synth.make_system(2, nwaters=4)
    g = kldi.make_grid(s.Z, s.xyz, s.grid.nrad, s.grid.ntheta)
    xyz, w, atom = g.export()
    blocks = [0, 11, g.nblocks // 3, g.nblocks - 1]
    go = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=blocks)
    sel = np.concatenate([np.arange(b * 128, (b + 1) * 128) for b in blocks])
    assert np.abs(xyz - go.points).max() < 1e-13
    assert np.abs(w[sel] - go.weights[sel]).max() < 1e-12


@pytest.fixture(scope="module")
def cnoh():
    return synth.make_system(3)


def test_cnoh1000_whole_grid_and_sampled_ranges(cnoh):
    import torch
    kldi = _kldi()
    s = cnoh
    plan = kldi.plan_for_system(s, prec="bf16x10", xc="pbe")
    nb = plan.stats["nblocks"]
    D = torch.from_numpy(s.D).cuda()

    def whole(prec):
        plan.set_precision(prec)
        V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        kldi.exc(plan, "pbe", D, V, E)
        torch.cuda.synchronize()
        return E.item(), V

    E10, V10 = whole("bf16x10")
    E6, V6 = whole("bf16x6")
    E64, V64 = whole("fp64")
    dV10 = (V10 - V64).abs().max().item()
    dV6 = (V6 - V64).abs().max().item()
    print(f"cnoh1000 whole grid: E_xc {E64:.9f} Ha (fp64); bf16x10 dE {E10 - E64:+.2e} max|dV| {dV10:.2e}; "
          f"bf16x6 dE {E6 - E64:+.2e} max|dV| {dV6:.2e}; max|V| {V64.abs().max().item():.3f}")
    assert np.isfinite(E64) and E64 < 0.0
    assert abs(E10 - E64) <= 1e-6
    assert dV10 <= 1e-7
    assert abs(E6 - E64) <= 5e-5            # BF16X6: its measured error, stated
    assert torch.equal(V10, V10.T)
    del V6
    # retained fraction of basis-block pairs (the workload's stated 5-15 % band)
    ptr, idx, _ = plan.lists()
    n = np.diff(ptr).astype(np.float64)
    frac = float(np.sum(n * n)) / (nb * plan.stats["nbasis_blocks"] ** 2)
    print(f"cnoh1000: mean retained blocks {n.mean():.1f} of {plan.stats['nbasis_blocks']}, "
          f"retained pair fraction {frac:.3f}")
    # sampled ranges against the oracle
    rng = np.random.default_rng(23)
    starts = sorted(rng.choice(nb - 6, size=3, replace=False).tolist())
    ranges = [(g0, g0 + 6) for g0 in starts]
    blocks = [b for g0, g1 in ranges for b in range(g0, g1)]
    go = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=blocks)
    sh = ob.build_shells(s.xyz, s.basis)
    rho_full = torch.zeros(plan.npoints, dtype=torch.float64, device="cuda")
    grad_full = torch.zeros((plan.npoints, 3), dtype=torch.float64, device="cuda")
    aD = np.abs(s.D)
    for g0, g1 in ranges:
        ref = oe.evaluate(s, go, sh, screened=True, blocks=range(g0, g1))
        pts = slice(g0 * 128, g1 * 128)
        ap = np.abs(ob.eval_basis(go.points[pts], sh, deriv=False)[0])
        bound = 2.0 ** -30 * (2.0 * ap.max(axis=1) * (ap @ aD.sum(axis=0)) + ap.sum(axis=1) * (ap @ aD.max(axis=0)))
        plan.set_block_range(g0, g1)        # work lists of the range only (cheap to switch precision)
        for prec, tE, tV in (("fp64", 1e-10, 1e-10), ("bf16x10", 1e-6, 1e-7)):
            plan.set_precision(prec)
            Vr = torch.zeros_like(V10)
            Er = torch.zeros(1, dtype=torch.float64, device="cuda")
            kldi.exc(plan, "pbe", D, Vr, Er)
            kldi.density(plan, D, rho_full, grad_full)
            torch.cuda.synchronize()
            r_gpu = rho_full[pts].cpu().numpy()
            dV = np.abs(Vr.cpu().numpy() - ref.V).max()
            ratio = np.abs(r_gpu - ref.rho[pts]) / (bound + 1e-300)
            print(f"range {g0} {prec}: dE {Er.item() - ref.E:.2e}, max|dV| {dV:.2e}, "
                  f"max rho error / bound {ratio.max():.3f}")
            assert abs(Er.item() - ref.E) <= tE, (g0, prec, Er.item(), ref.E)
            assert dV <= tV, (g0, prec, dV)
            if prec == "bf16x10":
                assert np.all(ratio <= 1.0), g0


def _density_points(system):
    kldi = _kldi()
    plan = kldi.plan_for_system(system, prec="fp64", xc="pbe")
    rho = np.zeros(plan.npoints)
    grad = np.zeros((plan.npoints, 3))
    kldi.density(plan, system.D, rho, grad)
    return rho, np.einsum("ic,ic->i", grad, grad)


def test_water167_learned_functional_fused():
    """The learned-functional workload: the network trained on the GPU on the
    grid points of the two-water and 33-water systems, fused between the
    products on the 167-water cluster (501 atoms, 4175 functions, 5.84M points).
    The whole-grid E_xc against the analytic functional is measured and
    stated; on seeded 6-block ranges the fused path is held to the oracle
    evaluating the same network (FP16 weights) at the learned functional's
    tolerances: |dE| <= 2e-5 sum |w e0|, max|dV| <= 2e-5 max|V| + 3e-7."""
    import torch
    from oracle import mlp as om
    kldi = _kldi()
    pts = [_density_points(synth.make_system(1)), _density_points(synth.make_system(2))]
    rho = np.concatenate([a for a, _ in pts])
    sig = np.concatenate([b for _, b in pts])
    box = synth.mlp_box(rho, sig)
    net = kldi.Mlp(synth.mlp_init(42), box)
    hist = net.train(rho, sig, epochs=100, batch=8192, lr0=3e-3, lr1=1e-5)
    assert hist[-1] < 1e-3 * hist[0]
    s = synth.make_system(5)
    plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe")
    D = torch.from_numpy(s.D).cuda()
    V = torch.zeros((s.nbf, s.nbf), dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    kldi.exc(plan, "pbe", D, V, E)
    E_pbe = E.item()
    kldi.plan_set_mlp(plan, net)
    kldi.exc(plan, "mlp", D, V, E)
    torch.cuda.synchronize()
    E_mlp = E.item()
    print(f"water167: E_xc analytic {E_pbe:.6f} Ha, learned {E_mlp:.6f} Ha, difference {E_mlp - E_pbe:.3e} Ha "
          f"({(E_mlp - E_pbe) / abs(E_pbe):.2e} relative)")
    assert abs(E_mlp - E_pbe) < 1e-3 * abs(E_pbe)
    nb = plan.stats["nblocks"]
    rng = np.random.default_rng(41)
    starts = sorted(rng.choice(nb - 6, size=2, replace=False).tolist())
    blocks = [b for g0 in starts for b in range(g0, g0 + 6)]
    go = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=blocks)
    sh = ob.build_shells(s.xyz, s.basis)
    p16 = om.fp16_weights(net.params())
    for g0 in starts:
        ref = oe.evaluate(s, go, sh, screened=True, blocks=range(g0, g0 + 6), xc_kind="mlp", mlp=(p16, om.Box(*box)))
        plan.set_block_range(g0, g0 + 6)
        Vr = torch.zeros_like(V)
        Er = torch.zeros_like(E)
        kldi.exc(plan, "mlp", D, Vr, Er)
        torch.cuda.synchronize()
        pts_ = slice(g0 * 128, (g0 + 6) * 128)
        e0 = np.abs(om.slater(np.maximum(ref.rho[pts_], 1e-300))[0]) * (ref.rho[pts_] >= 1e-14)
        scaleE = float(np.sum(np.abs(go.weights[pts_]) * e0))
        dV = np.abs(Vr.cpu().numpy() - ref.V).max()
        print(f"range {g0}: dE {Er.item() - ref.E:.2e} (bound {2e-5 * scaleE:.1e}), max|dV| {dV:.2e}")
        assert abs(Er.item() - ref.E) <= 2e-5 * scaleE
        assert dV <= 2e-5 * np.abs(ref.V).max() + 3e-7

"""GPU parity of the learned functional (forward with its input derivative,
loss gradient, Adam step, fused quadrature) against the FP64 oracle in
oracle/mlp.py, and what training gains.

Tolerances (FP32 network arithmetic on FP16 weights; the oracle uses the same
FP16 values in FP64): every pre-activation sums 64 products of magnitude
<= ~1, so outputs carry ~64 x 2^-24 ~ 4e-6 absolute error at worst:
  f, v_rho       |d| <= 2e-5 x |e0|, |v0|   (e0, v0: Slater energy density, potential)
  v_sigma        |d| <= 2e-5 x |e0| / (s2 sigma)
  loss, grad     relative 1e-4 (sums of 1e3..1e4 per-point FP32 terms)
  Adam step      relative 1e-5 (FP32 update of the same gradient)
  quadrature     |dE| <= 2e-5 x sum_i |w_i e0_i|, max|dV| <= 2e-5 x max|V| + 3e-7
"""
import math

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og
from oracle import mlp as om
from oracle import xc as ox

pytestmark = pytest.mark.gpu


def _kldi():
    from paper_2605_10363_gb300 import kldi
    return kldi


def _points(n=4000, seed=11):
    rho, sigma = synth.mlp_points(n, seed)
    rho[:7] = [1e-15, 1e-13, 2e-12, 1e-11, 5e3, 1e-3, 1e-3]      # below rho_min, outside the box, inside
    sigma[5] = 0.0
    sigma[6] = 1e-40
    return rho, sigma


def test_eval_matches_oracle():
    kldi = _kldi()
    rho, sigma = _points()
    p = synth.mlp_init(7)
    box = synth.mlp_box(*synth.mlp_points(4000, 11))
    net = kldi.Mlp(p, box)
    f, vr, vs, used = net.eval(rho, sigma)
    fo, vro, vso, usedo = om.functional(om.fp16_weights(p), om.Box(*box), rho, sigma)
    assert np.array_equal(used, usedo)
    e0, v0 = om.slater(rho)
    s2 = 0.5 * (box[3] - box[2])
    sig = np.maximum(sigma, om.SIGMA_FLOOR)
    assert np.all(np.abs(f - fo) <= 2e-5 * np.abs(e0))
    assert np.all(np.abs(vr - vro) <= 2e-5 * np.abs(v0))
    assert np.all(np.abs(vs - vso) <= 2e-5 * np.abs(e0) / (s2 * sig))
    # fallback points agree with the analytic functional to FP64 rounding
    fa, vra, vsa = ox.evaluate("pbe", rho, sigma)
    out = ~used & (rho >= 1e-14)
    assert out.sum() >= 3
    assert np.allclose(f[out], fa[out], rtol=1e-12, atol=0)
    assert np.all(f[rho < 1e-14] == 0.0)


def test_loss_grad_matches_oracle():
    kldi = _kldi()
    rho, sigma = _points(3000, 13)
    p = synth.mlp_init(9)
    box = synth.mlp_box(rho[7:], sigma[7:])
    net = kldi.Mlp(p, box)
    loss, g = net.loss_grad(rho, sigma)
    p16 = om.fp16_weights(p)
    B = om.Box(*box)
    z, inside = om.inputs(np.maximum(rho, 1e-300), sigma, B)
    ok = inside & (rho >= 1e-14)
    tF, tG = np.zeros(rho.size), np.zeros(rho.size)
    tF[ok], tG[ok] = om.targets(rho[ok], sigma[ok])
    z[~ok] = 0.0
    lo, go = om.loss_grad(p16, z, tF, tG, ok.astype(float))
    assert loss == pytest.approx(lo, rel=1e-4)
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go) + 1e-5 * np.abs(go).max())


def test_adam_step_matches_oracle():
    kldi = _kldi()
    p = synth.mlp_init(3)
    box = np.array([-20.0, 5.0, -60.0, 20.0])
    net = kldi.Mlp(p, box)
    rng = np.random.default_rng(4)
    po, m, v = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    for t in range(1, 4):
        g = rng.normal(size=p.size).astype(np.float32) * 10.0 ** rng.uniform(-4, 0, size=p.size).astype(np.float32)
        net.adam_step(g, 1e-3)
        po, m, v = om.adam(po, m, v, g.astype(np.float64), t, 1e-3)
    got = net.params()
    assert np.all(np.abs(got - po) <= 1e-5 * np.abs(po) + 1e-9)


def _density_points(system):
    kldi = _kldi()
    plan = kldi.plan_for_system(system, prec="fp64", xc="pbe")
    rho = np.zeros(plan.npoints)
    grad = np.zeros((plan.npoints, 3))
    kldi.density(plan, system.D, rho, grad)
    return rho, np.einsum("ic,ic->i", grad, grad)


@pytest.fixture(scope="module")
def trained():
    """A network trained on the GPU on the densities of the two-water and
    four-water systems (the method's own grid points)."""
    kldi = _kldi()
    pts = [_density_points(synth.make_system(1)), _density_points(synth.make_system(2, nwaters=4))]
    rho = np.concatenate([a for a, _ in pts])
    sigma = np.concatenate([b for _, b in pts])
    box = synth.mlp_box(rho, sigma)
    net = kldi.Mlp(synth.mlp_init(42), box)
    hist = net.train(rho, sigma, epochs=300, batch=4096, lr0=3e-3, lr1=1e-5)
    return net, box, hist


def test_checkpoint_resumes_training_bit_for_bit():
    """The training state (parameters, Adam moments, step counter) saved after
    some epochs and restored into a fresh network gives exactly the same
    parameters and losses after the same further training."""
    kldi = _kldi()
    rho, sigma = _density_points(synth.make_system(1))
    box = synth.mlp_box(rho, sigma)
    net = kldi.Mlp(synth.mlp_init(42), box)
    net.train(rho, sigma, epochs=3, batch=2048)
    state, step = net.state()
    assert step > 0 and np.all(np.isfinite(state))
    assert np.array_equal(state[:kldi.MLP_NPARAMS], net.params())
    h1 = net.train(rho, sigma, epochs=2, batch=2048)
    p1 = net.params()
    other = kldi.Mlp(synth.mlp_init(7), box)
    other.set_state(state, step)
    s2, step2 = other.state()
    assert step2 == step and np.array_equal(s2, state)
    h2 = other.train(rho, sigma, epochs=2, batch=2048)
    assert np.array_equal(h1, h2)
    assert np.array_equal(p1, other.params())
    with pytest.raises(kldi.KldiError):
        other.set_state(state, -1)


def test_training_reduces_loss(trained):
    net, box, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 1e-3 * hist[0], hist


def test_fused_quadrature_matches_oracle_with_same_network(trained):
    kldi = _kldi()
    net, box, _ = trained
    s = synth.make_system(1)
    p16 = om.fp16_weights(net.params())
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    ref = oe.evaluate(s, g, sh, screened=True, xc_kind="mlp", mlp=(p16, om.Box(*box)))
    e0 = np.abs(om.slater(np.maximum(ref.rho, 1e-300))[0])
    scaleE = float(np.sum(np.abs(g.weights) * e0 * (ref.rho >= 1e-14)))
    for prec, tv in (("fp64", 0.0), ("bf16x6", 3e-7)):
        plan = kldi.plan_for_system(s, prec=prec, xc="pbe")
        kldi.plan_set_mlp(plan, net)
        V = np.zeros((s.nbf, s.nbf))
        E = np.zeros(1)
        kldi.exc(plan, "mlp", s.D, V, E)
        assert abs(E[0] - ref.E) <= 2e-5 * scaleE, (prec, E[0], ref.E)
        assert np.abs(V - ref.V).max() <= 2e-5 * np.abs(ref.V).max() + tv, prec
        assert np.array_equal(V, V.T)


def test_mlp_call_needs_network():
    kldi = _kldi()
    s = synth.make_system(1)
    plan = kldi.plan_for_system(s, prec="fp64", xc="pbe")
    with pytest.raises(kldi.KldiError) as e:
        kldi.exc(plan, "mlp", s.D, np.zeros((s.nbf, s.nbf)), np.zeros(1))
    assert e.value.status == kldi.EINVAL
    lda = kldi.plan_for_system(s, prec="fp64", xc="lda_x")
    net = kldi.Mlp(synth.mlp_init(1), np.array([-30.0, 5.0, -69.0, 20.0]))
    with pytest.raises(kldi.KldiError):
        kldi.plan_set_mlp(lda, net)


def test_what_training_gains(trained):
    """The learned functional against the method without it, the analytic
    PBE-form path (the reference), on the four-water system: the E_xc difference
    and the time of the whole evaluation and of the functional stage are
    measured and stated; the trained network's difference is bounded (1e-3
    relative) and more than 20x smaller than that of the untrained network
    (Slater exchange), which shows what the training adds."""
    kldi = _kldi()
    net, box, _ = trained
    s = synth.make_system(2, nwaters=4)
    E_of, stage_ms, total_ms = {}, {}, {}
    for name, netw in (("analytic", None), ("trained", net), ("untrained", kldi.Mlp(synth.mlp_init(42), box))):
        plan = kldi.plan_for_system(s, prec="bf16x6", xc="pbe")
        xc = "pbe"
        if netw is not None:
            kldi.plan_set_mlp(plan, netw)
            xc = "mlp"
        V = np.zeros((s.nbf, s.nbf))
        E = np.zeros(1)
        kldi.exc(plan, xc, s.D, V, E)
        plan.profile(True)
        for _ in range(5):
            kldi.exc(plan, xc, s.D, V, E)
        ms, _ = plan.stage_times()
        stage_ms[name] = ms[3] / 5
        total_ms[name] = ms.sum() / 5
        E_of[name] = E[0]
    d_tr = abs(E_of["trained"] - E_of["analytic"])
    d_un = abs(E_of["untrained"] - E_of["analytic"])
    print(f"learned vs analytic: dE {d_tr:.3e} Ha ({d_tr / abs(E_of['analytic']):.1e} relative), "
          f"evaluation {total_ms['trained']:.3f} ms vs {total_ms['analytic']:.3f} ms, "
          f"functional stage {stage_ms['trained']:.4f} ms vs {stage_ms['analytic']:.4f} ms; "
          f"untrained network dE {d_un:.3e} Ha")
    assert d_tr <= 1e-3 * abs(E_of["analytic"])
    assert d_tr < d_un / 20.0


def test_gradient_with_learned_functional(trained):
    """Nuclear gradient with the fused network: the X coefficients a, b come from
    the FP32 network (relative error <= 2e-5 of the Slater scale, above), and
    the gradient is linear in them, so |dG| <= 2e-5 Gmag (the oracle's term
    magnitudes) in both the FP64 and the BF16x6 forms."""
    from oracle import grad as ogr
    kldi = _kldi()
    net, box, _ = trained
    s = synth.make_system(1)
    p16 = om.fp16_weights(net.params())
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    Gref, Gmag = ogr.exc_gradient(s, g, sh, screened=True, xc_kind="mlp", mlp=(p16, om.Box(*box)),
                                  return_magnitude=True)
    for prec in ("fp64", "bf16x6"):
        plan = kldi.plan_for_system(s, prec=prec, xc="pbe")
        kldi.plan_set_mlp(plan, net)
        G = np.zeros((len(s.Z), 3))
        E = np.zeros(1)
        kldi.exc_grad(plan, "mlp", s.D, G, E)
        d = np.abs(G - Gref)
        print(f"learned functional gradient {prec}: max|dG| {d.max():.2e}, max dG/Gmag {(d / Gmag).max():.2e}")
        assert np.all(d <= 2e-5 * Gmag), prec

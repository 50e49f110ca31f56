"""Pins of the FP64 surrogate oracle (oracle/mlp.py) against finite
differences, closed forms and degenerate cases; no GPU."""
import math

import numpy as np
import pytest

import synth
from oracle import mlp as om
from oracle import xc as ox


def _setup(n=40, seed=3):
    p = om.fp16_weights(synth.mlp_init(seed))
    rho, sigma = synth.mlp_points(n, seed)
    box = om.Box(*synth.mlp_box(rho, sigma))
    z, inside = om.inputs(rho, sigma, box)
    return p, rho, sigma, box, z, inside


def test_parameter_layout():
    assert om.NP == synth.MLP_NPARAMS == 4482
    W1, b1, W2, b2, W3, b3 = om.unpack(np.arange(om.NP, dtype=float))
    assert W1.shape == (64, 2) and W2.shape == (64, 64) and W3.shape == (2, 64)
    assert b3[1] == om.NP - 1


def test_backward_matches_finite_differences():
    p, rho, sigma, box, z, _ = _setup()
    tF, tG = om.targets(rho, sigma)
    mask = np.ones(rho.size)
    mask[::7] = 0.0                                   # masked points must not contribute
    loss, g = om.loss_grad(p, z, tF, tG, mask)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.arange(om.O_W1, om.O_B1), 6), rng.choice(np.arange(om.O_B1, om.O_W2), 4),
                          rng.choice(np.arange(om.O_W2, om.O_B2), 10), rng.choice(np.arange(om.O_B2, om.O_W3), 4),
                          rng.choice(np.arange(om.O_W3, om.O_B3), 6), np.arange(om.O_B3, om.NP)])
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (om.loss_grad(pp, z, tF, tG, mask)[0] - om.loss_grad(pm, z, tF, tG, mask)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_input_derivative_and_v_sigma_match_finite_differences():
    p, rho, sigma, box, z, inside = _setup(60, 5)
    o, cache = om.forward(p, z)
    d = om.do1_dz2(p, cache)
    h = 1e-6
    zp, zm = z.copy(), z.copy()
    zp[:, 1] += h
    zm[:, 1] -= h
    fd = (om.forward(p, zp)[0][:, 0] - om.forward(p, zm)[0][:, 0]) / (2 * h)
    assert np.allclose(d, fd, rtol=1e-7, atol=1e-9)
    # v_sigma is df/dsigma of the network's energy density (inside the box)
    sel = np.where(np.all(np.abs(z) < 0.99, axis=1) & (sigma > 1e-28))[0][:20]   # away from the box edge
    r, s = rho[sel], sigma[sel]
    f, vr, vs, net = om.functional(p, box, r, s)
    assert net.all()
    hs = 1e-4 * s
    fp = om.functional(p, box, r, s + hs)[0]
    fm = om.functional(p, box, r, s - hs)[0]
    # central difference: truncation ~1e-8 relative, rounding ~1e-16 |f| / hs
    assert np.all(np.abs(vs - (fp - fm) / (2 * hs)) <= 1e-6 * np.abs(vs) + 1e-11 * np.abs(f) / hs)


def test_targets_at_zero_gradient_are_slater_plus_pw92():
    rho = np.exp(np.linspace(math.log(1e-6), math.log(1e2), 25))
    F, G = om.targets(rho, np.zeros_like(rho))
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    e0 = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * rho ** (4.0 / 3.0)
    assert np.allclose(F, 1.0 + rho * ox.eps_pw92(rs) / e0, rtol=1e-12)
    # G at sigma = 0: exchange part is exactly 1
    _, vr_x = ox.evaluate("lda_x", rho, None, 0.0)[:2]
    assert np.allclose(vr_x / om.slater(rho)[1], 1.0, rtol=1e-12)
    assert np.all(G > 1.0)


def test_degenerate_weights():
    p = np.zeros(om.NP)
    p[om.O_B3:] = [1.25, 0.75]
    rho, sigma = synth.mlp_points(30, 9)
    box = om.Box(*synth.mlp_box(rho, sigma))
    f, vr, vs, net = om.functional(p, box, rho, sigma)
    e0, v0 = om.slater(rho)
    assert np.allclose(f[net], 1.25 * e0[net], rtol=1e-14)
    assert np.allclose(vr[net], 0.75 * v0[net], rtol=1e-14)
    assert np.all(vs[net] == 0.0)
    # outside the box the analytic functional is used
    out = np.array([1e-13]), np.array([1e-20])
    f1, vr1, vs1, net1 = om.functional(p, box, *out)
    fa, vra, vsa = ox.evaluate("pbe", *out)
    assert not net1[0] and f1[0] == fa[0] and vs1[0] == vsa[0]
    # below rho_min nothing
    f2 = om.functional(p, box, np.array([1e-15]), np.array([1e-30]))[0]
    assert f2[0] == 0.0


def test_adam_first_step_and_convergence():
    g = np.array([3.0, -0.5, 1e-3])
    p1, m, v = om.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), rtol=1e-4)
    # Adam on 0.5 * a * p^2 reaches the minimum
    a = np.array([1.0, 10.0, 0.1])
    p, m, v = np.array([1.0, -2.0, 3.0]), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        p, m, v = om.adam(p, m, v, a * p, t, om.cosine_lr(t - 1, 3000, 0.05, 1e-4))
    assert np.all(np.abs(p) < 1e-2)


def test_fp16_weights_round_to_half():
    p = synth.mlp_init(1)
    q = om.fp16_weights(p)
    assert np.all(q.astype(np.float16).astype(np.float64) == q)
    assert np.max(np.abs(q - p)) <= 2.0 ** -11 * np.max(np.abs(p))


def test_cosine_schedule_endpoints():
    assert om.cosine_lr(0, 100, 1e-2, 1e-4) == pytest.approx(1e-2)
    assert om.cosine_lr(99, 100, 1e-2, 1e-4) == pytest.approx(1e-4)


def test_quadrature_with_constant_network_is_slater_exchange():
    """W = 0, b3 = (1, 1) over a box holding every point: f = e0 and
    v_rho = v0, v_sigma = 0, so E and V equal the Slater-exchange quadrature."""
    from oracle import basis as ob
    from oracle import exc as oe
    from oracle import grid as og
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    p = np.zeros(om.NP)
    p[om.O_B3:] = 1.0
    box = om.Box(math.log(1e-14), math.log(1e6), math.log(1e-30), math.log(1e12))
    r1 = oe.evaluate(s, g, sh, screened=True, xc_kind="mlp", mlp=(p, box))
    r0 = oe.evaluate(s, g, sh, screened=True, xc_kind="lda_x")
    assert r1.E == pytest.approx(r0.E, rel=1e-13)
    assert np.abs(r1.V - r0.V).max() <= 1e-12

"""Pins of the FP64 nuclear-gradient oracle (oracle/grad.py)."""
import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grad as og_
from oracle import grid as og


def test_basis_hessian_matches_finite_differences_of_gradient():
    s = synth.make_system(2, nwaters=1)                  # s, p and d shells
    sh = ob.build_shells(s.xyz, s.basis)
    rng = np.random.default_rng(3)
    pts = s.xyz[rng.integers(0, 3, 12)] + rng.normal(scale=0.7, size=(12, 3))
    phi, dphi, hphi = og_.eval_basis_hessian(pts, sh)
    phi0, dphi0 = ob.eval_basis(pts, sh, deriv=True)
    assert np.allclose(phi, phi0, rtol=1e-14, atol=1e-300) and np.allclose(dphi, dphi0, rtol=1e-13, atol=1e-300)
    h = 1e-5
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        fd = (ob.eval_basis(pts + e, sh, deriv=True)[1] - ob.eval_basis(pts - e, sh, deriv=True)[1]) / (2 * h)
        assert np.allclose(hphi[:, b], fd, rtol=1e-6, atol=1e-8 * np.abs(hphi).max())
    assert np.allclose(hphi, np.swapaxes(hphi, 0, 1))


def _fd_gradient(s, grid, kind, atom, axis, h=1e-4):
    def energy(delta):
        xyz = s.xyz.copy()
        xyz[atom, axis] += delta
        sh = ob.build_shells(xyz, s.basis)
        return oe.evaluate(s, grid, sh, screened=False, want_v=False, xc_kind=kind).E
    return (energy(h) - energy(-h)) / (2 * h)


@pytest.mark.parametrize("kind", ["lda_x", "pbe"])
def test_gradient_matches_finite_differences_on_fixed_grid(kind):
    s = synth.make_system(2, nwaters=1) if kind == "pbe" else synth.make_system(1)
    grid = og.build_grid(s.Z, s.xyz, s.grid)
    G = og_.exc_gradient(s, grid, screened=False, xc_kind=kind)
    for atom, axis in ((0, 0), (1, 2), (len(s.Z) - 1, 1)):
        fd = _fd_gradient(s, grid, kind, atom, axis)
        assert abs(fd - G[atom, axis]) <= 1e-7 + 1e-5 * abs(fd), (kind, atom, axis, fd, G[atom, axis])


def test_screened_gradient_at_zero_thresholds_is_dense():
    s = synth.make_system(1)
    grid = og.build_grid(s.Z, s.xyz, s.grid)
    Gd = og_.exc_gradient(s, grid, screened=False, xc_kind="pbe")
    Gs = og_.exc_gradient(s, grid, screened=True, xc_kind="pbe", t_b=0.0, t_d=0.0)
    assert np.allclose(Gs, Gd, rtol=1e-12, atol=1e-14)


def test_gradient_with_learned_functional_matches_finite_differences():
    """The gradient is formed from the functional's (f, v_rho, v_sigma); the
    surrogate's v_rho is a separate network output (trained towards the
    analytic one), so the formula is the derivative of E only when that output
    is df/drho.  A network with zero weights and equal output biases c is
    exactly that (f = c e0, v_rho = c v0 = df/drho, v_sigma = 0): the oracle's
    gradient through the network path must then match finite differences."""
    import math

    from oracle import mlp as om
    s = synth.make_system(1)
    grid = og.build_grid(s.Z, s.xyz, s.grid)
    p = np.zeros(om.NP)
    p[om.O_B3:] = 1.3
    box = om.Box(math.log(1e-14) - 1.0, math.log(1e6), math.log(1e-30) - 1.0, math.log(1e12))
    mlp = (p, box)
    G = og_.exc_gradient(s, grid, screened=False, xc_kind="mlp", mlp=mlp)
    Gx = og_.exc_gradient(s, grid, screened=False, xc_kind="lda_x")
    assert np.allclose(G, 1.3 * Gx, rtol=1e-12, atol=1e-15)      # the network is 1.3 x Slater exchange

    def energy(atom, axis, delta):
        xyz = s.xyz.copy()
        xyz[atom, axis] += delta
        return oe.evaluate(s, grid, ob.build_shells(xyz, s.basis), screened=False, want_v=False, xc_kind="mlp",
                           mlp=mlp).E

    h = 1e-4
    for atom, axis in ((0, 1), (4, 0)):
        fd = (energy(atom, axis, h) - energy(atom, axis, -h)) / (2 * h)
        assert abs(fd - G[atom, axis]) <= 1e-7 + 1e-5 * abs(fd), (atom, axis, fd, G[atom, axis])

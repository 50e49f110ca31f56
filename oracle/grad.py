"""Nuclear gradient of E_xc (the paper's second workload: "energies and
gradients", Sec. IV, Fig. 4), FP64 reference.

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline use this module; the library never calls it.

Reading (the paper names the gradient but prints no formula): the derivative
of E_xc = sum_i w_i f(rho_i, sigma_i) with respect to the position R_A of
atom A through the basis functions centred on A, on a fixed grid (points and
weights do not move: no grid-weight response).  With chi_mu centred on
A(mu), d chi_mu / d R_A = -grad chi_mu for mu on A, and D fixed:

  dE/dR_A,x = -2 sum_{mu on A} sum_i [ d_x chi_mu(r_i) Q_mu,i
                                       + (b_i . grad d_x chi_mu(r_i)) R_mu,i ]

  R = Phi D,  Q = Z D,  Z_nu,i = w_i v_rho,i chi_nu,i + 2 w_i v_sigma,i grad rho_i . grad chi_nu,i,
  b_i = 2 w_i v_sigma,i grad rho_i

(LDA: v_sigma = 0, so only the first term remains).  The screened form
restricts both products R and Q to the executed block pairs E1_g of the
density product (they are products with D), as oracle.exc does for R.

Pins (tests/test_oracle_grad.py): the basis Hessian against central
differences of the analytic first derivatives; the gradient (dense, LDA and
GGA) against central differences of E_xc with the basis centres of one atom
displaced on the fixed grid; the screened gradient at zero thresholds equals
the dense one.
"""
from __future__ import annotations

import numpy as np

from . import basis as obasis
from . import exc as oexc
from . import screen as oscreen
from . import xc as oxc


def _mono(d, comp, dp):
    """prod_c d_c^(comp_c - dp_c) * falling-factorial coefficients: the
    derivative of x^i y^j z^k of orders dp (per axis)."""
    out = np.ones(d.shape[0])
    for ax in range(3):
        p, k = comp[ax], dp[ax]
        if k > p:
            return np.zeros(d.shape[0])
        coef = 1.0
        for t in range(k):
            coef *= (p - t)
        out = out * coef * d[:, ax] ** (p - k)
    return out


def eval_basis_hessian(points: np.ndarray, shells: list):
    """phi [i, mu], dphi [a, i, mu] and the Hessian hphi [a, b, i, mu] =
    d^2 chi_mu / dr_a dr_b of the contracted Cartesian Gaussians:
    chi = P g, g = sum c e^{-alpha r^2}, G1 = sum c alpha e^{-alpha r^2},
    G2 = sum c alpha^2 e^{-alpha r^2}:
      d_a chi = (d_a P) g - 2 d_a P G1
      d_a d_b chi = (d_a d_b P) g - 2 (d_a P r_b + d_b P r_a) G1 + P (4 r_a r_b G2 - 2 delta_ab G1)."""
    npts = points.shape[0]
    nbf = sum(s.size for s in shells)
    phi = np.zeros((npts, nbf))
    dphi = np.zeros((3, npts, nbf))
    hphi = np.zeros((3, 3, npts, nbf))
    eye = np.eye(3, dtype=int)
    mu = 0
    for sh in shells:
        d = points - sh.center
        r2 = np.einsum("ij,ij->i", d, d)
        e = np.exp(-np.outer(r2, sh.exps))
        for comp, c in zip(sh.components, sh.coefs):
            g = e @ c
            g1 = e @ (c * sh.exps)
            g2 = e @ (c * sh.exps ** 2)
            P = _mono(d, comp, (0, 0, 0))
            dP = [_mono(d, comp, tuple(eye[a])) for a in range(3)]
            phi[:, mu] = P * g
            for a in range(3):
                dphi[a, :, mu] = dP[a] * g - 2.0 * d[:, a] * P * g1
                for b in range(3):
                    ddP = _mono(d, comp, tuple(eye[a] + eye[b]))
                    hphi[a, b, :, mu] = (ddP * g - 2.0 * (dP[a] * d[:, b] + dP[b] * d[:, a]) * g1
                                         + P * (4.0 * d[:, a] * d[:, b] * g2 - (2.0 * g1 if a == b else 0.0)))
            mu += 1
    return phi, dphi, hphi


def function_atoms(system) -> np.ndarray:
    """Atom index of every basis function (basis-function order)."""
    out = []
    for s in range(len(system.basis.atom)):
        out += [int(system.basis.atom[s])] * ((system.basis.l[s] + 1) * (system.basis.l[s] + 2) // 2)
    return np.array(out, dtype=np.int64)


def exc_gradient(system, grid, shells=None, screened=True, xc_kind=None, t_b=None, t_d=None,
                 rho_min=oxc.RHO_MIN, mlp=None, return_magnitude=False, blocks=None):
    """dE_xc/dR_A (natm x 3) on the fixed grid, the formula of the module docstring.
    With return_magnitude, also the sums of the terms' magnitudes per atom and
    component, 2 sum_{mu on A} sum_i (|d_x chi Q| + |b . grad d_x chi| |R|): the
    scale against which rounding errors of the terms are measured.  `blocks`
    restricts the sum to those grid blocks (a rank's share of the grid)."""
    from . import mlp as omlp
    if shells is None:
        shells = obasis.build_shells(system.xyz, system.basis)
    kind = xc_kind or system.xc
    gga = kind in ("pbe", "mlp")
    t_b = system.t_b if t_b is None else t_b
    t_d = system.t_d if t_d is None else t_d
    D = system.D
    nbf = D.shape[0]
    fatom = function_atoms(system)
    natm = len(system.Z)
    G = np.zeros((natm, 3))
    Gmag = np.zeros((natm, 3))
    dmax = oscreen.d_block_max(D)
    dsz = oscreen.D_BASIS
    nb = oscreen.nbasis_blocks(nbf)
    B = grid.block
    for g in (range(grid.nblocks) if blocks is None else blocks):
        sl = slice(g * B, (g + 1) * B)
        pts = grid.points[sl]
        w = grid.weights[sl]
        phi, dphi, hphi = eval_basis_hessian(pts, shells)
        if screened:
            summ = np.abs(phi)
            if gga:
                summ = np.maximum(summ, np.abs(dphi).max(axis=0))
            b = oscreen.block_max_cols(summ)
            S = oscreen.retained(b, t_b)
        else:
            b = np.ones(nb)
            S = np.arange(nb)
        if S.size == 0:
            continue
        cols = np.concatenate([np.arange(p * dsz, min((p + 1) * dsz, nbf)) for p in S])
        pos = {int(p): i for i, p in enumerate(S)}
        cb = np.array([pos[int(c)] for c in cols // dsz], dtype=np.int64)
        Dg = D[np.ix_(cols, cols)].copy()
        if screened:
            E1 = oscreen.executed_rho(S, b, dmax, t_b, t_d)
            Dg *= E1[np.ix_(cb, cb)]
        ph = phi[:, cols]
        dph = dphi[:, :, cols]
        hph = hphi[:, :, :, cols]
        R = ph @ Dg
        rho = np.einsum("im,im->i", ph, R)
        if gga:
            grad = 2.0 * np.einsum("cim,im->ic", dph, R)
            sigma = np.einsum("ic,ic->i", grad, grad)
        else:
            grad = np.zeros((pts.shape[0], 3))
            sigma = None
        if kind == "mlp":
            f, vr, vs, _ = omlp.functional(mlp[0], mlp[1], rho, sigma, rho_min)
        else:
            f, vr, vs = oxc.evaluate(kind, rho, sigma, rho_min)
        bvec = (2.0 * w * vs)[:, None] * grad                       # b_i
        Z = (w * vr)[:, None] * ph + np.einsum("ic,cim->im", bvec, dph)
        Q = Z @ Dg
        # per function: sum_i d_x chi Q + (b . grad d_x chi) R
        t1 = np.einsum("xim,im->xm", dph, Q)
        t2 = np.einsum("ic,xcim,im->xm", bvec, hph, R)
        contrib = -2.0 * (t1 + t2)                                   # [3, n_cols]
        np.add.at(G, fatom[cols], contrib.T)
        if return_magnitude:
            m1 = np.einsum("xim,im->xm", np.abs(dph), np.abs(Q))
            m2 = np.einsum("xim,im->xm", np.abs(np.einsum("ic,xcim->xim", bvec, hph)), np.abs(R))
            np.add.at(Gmag, fatom[cols], (2.0 * (m1 + m2)).T)
    return (G, Gmag) if return_magnitude else G

"""Exchange-correlation quadrature: rho, E_xc and V_xc, dense and screened.

Definitions followed (paper Sec. II-A and App. A):
  Phi_{mu i} = chi_mu(r_i)                                   (Eq. phi_def)
  rho_i = sum_{mu nu} D_{mu nu} chi_mu(r_i) chi_nu(r_i)      (App. A, "The density matrix")
        = sum_mu Phi_{mu i} R_{mu i},  R = D Phi              (Eq. r_equals_dphi)
  grad rho_i = 2 sum_{mu nu} D_{mu nu} grad chi_mu chi_nu     (GGA, D symmetric)
  E_xc = sum_i w_i f(rho_i, sigma_i)
  F^xc_{mu nu} = b sum_i w_i v_i chi_mu chi_nu, b = 1         (Eq. exc_quadrature, Eq. fxc_matrix_form)
and for the GGA the standard semilocal generalisation
  V_{mu nu} = sum_i w_i [v_rho chi_mu chi_nu + 2 v_sigma grad rho . (grad chi_mu chi_nu + chi_mu grad chi_nu)]
            = (Phi^T X + X^T Phi)_{mu nu},
  X_{i nu}  = w_i (v_rho chi_nu / 2 + 2 v_sigma grad rho_i . grad chi_nu(r_i)).
(For LDA this is X = W Phi^T / 2 with W = diag(w v), Eq. w_def.)

The screened form restricts every product to the executed block pairs of
``oracle.screen`` (Eq. executed_block_output): non-executed 32 x 32 blocks of D
(for R) contribute nothing, and a block (p, q) of a grid block's
Phi^T X + X^T Phi is added, both terms, when (p, q) or (q, p) is an executed
pair of the potential product.  The dense form keeps all.

Pins (tests): the closed-form Slater exchange energy of one doubly occupied
normalised s-Gaussian; sum w rho = tr(D S); V = V^T; tr(D V) = 4/3 E_x for
Slater exchange; tr(D V) = sum w (rho v_rho + 2 sigma v_sigma) for the GGA;
E_x[lambda D] = lambda^(4/3) E_x[D]; dE_xc/dD = V by central differences;
dense against an einsum of the definition on a tiny case; screened equals
dense when every pair is kept, and the screened-dense gap is within the
threshold bound.
"""
from __future__ import annotations

import numpy as np

from . import basis as obasis
from . import mlp as omlp
from . import screen as oscreen
from . import xc as oxc


class Result:
    def __init__(self, nbf, npts):
        self.rho = np.zeros(npts)
        self.grad = np.zeros((npts, 3))
        self.exc_blocks = None
        self.E = 0.0
        self.V = np.zeros((nbf, nbf))
        self.lists = {}


def _block_phi(shells, points, gga):
    phi, dphi = obasis.eval_basis(points, shells, deriv=gga)
    return phi, dphi


def evaluate(system, grid, shells=None, screened=True, blocks=None, want_v=True,
             keep_lists=False, xc_kind=None, t_b=None, t_d=None, rho_min=oxc.RHO_MIN, mlp=None):
    """rho, grad rho, E_xc and V over the grid blocks ``blocks`` (default all).

    With a subset of blocks, E and V are the partial sums over those blocks.
    ``xc_kind="mlp"`` uses the learned functional ``mlp = (fp16 weights, Box)``
    of oracle.mlp (a GGA: it needs grad rho)."""
    if shells is None:
        shells = obasis.build_shells(system.xyz, system.basis)
    kind = xc_kind or system.xc
    gga = kind in ("pbe", "mlp")
    t_b = system.t_b if t_b is None else t_b
    t_d = system.t_d if t_d is None else t_d
    D = system.D
    nbf = D.shape[0]
    B = grid.block
    if blocks is None:
        blocks = range(grid.nblocks)
    blocks = list(blocks)
    res = Result(nbf, grid.npoints)
    res.exc_blocks = np.zeros(len(blocks))
    dmax = oscreen.d_block_max(D)
    d = oscreen.D_BASIS
    nb = oscreen.nbasis_blocks(nbf)
    for k, g in enumerate(blocks):
        sl = slice(g * B, (g + 1) * B)
        pts = grid.points[sl]
        w = grid.weights[sl]
        phi, dphi = _block_phi(shells, pts, gga)
        if screened:
            summ = np.abs(phi)
            if gga:
                summ = np.maximum(summ, np.abs(dphi).max(axis=0))
            b = oscreen.block_max_cols(summ)
            S = oscreen.retained(b, t_b)
        else:
            b = np.ones(nb)
            S = np.arange(nb)
        cols = np.concatenate([np.arange(p * d, min((p + 1) * d, nbf)) for p in S]) if S.size else np.zeros(0, int)
        # block index of every retained column
        colblk = cols // d
        pos = {int(p): i for i, p in enumerate(S)}
        cb = np.array([pos[int(c)] for c in colblk], dtype=np.int64)
        # --- R = Phi_g D over executed pairs (Eq. executed_block_output)
        Dg = D[np.ix_(cols, cols)].copy()
        if screened:
            E1 = oscreen.executed_rho(S, b, dmax, t_b, t_d)
            Dg *= E1[np.ix_(cb, cb)]
        else:
            E1 = np.ones((S.size, S.size), dtype=bool)
        ph = phi[:, cols]
        R = ph @ Dg
        rho = np.einsum("im,im->i", ph, R)
        res.rho[sl] = rho
        if gga:
            dph = dphi[:, :, cols]
            grad = 2.0 * np.einsum("cim,im->ic", dph, R)
            res.grad[sl] = grad
            sigma = np.einsum("ic,ic->i", grad, grad)
        else:
            dph = None
            sigma = None
        if kind == "mlp":
            f, vr, vs, _ = omlp.functional(mlp[0], mlp[1], rho, sigma, rho_min)
        else:
            f, vr, vs = oxc.evaluate(kind, rho, sigma, rho_min)
        eg = float(np.sum(w * f))
        res.exc_blocks[k] = eg
        res.E += eg
        if keep_lists:
            res.lists[g] = {"S": S.copy(), "b": b.copy(), "E1": E1.copy()}
        if not want_v or S.size == 0:
            continue
        # --- X and V += Phi^T X + X^T Phi over executed pairs
        X = 0.5 * (w * vr)[:, None] * ph
        if gga:
            X += 2.0 * (w * vs)[:, None] * np.einsum("ic,cim->im", grad, dph)
        Vg = ph.T @ X
        Vg = Vg + Vg.T
        if screened:
            x = np.zeros(nb)
            ax = np.abs(X)
            for i, p in enumerate(S):
                x[p] = ax[:, cb == i].max()
            E2 = oscreen.executed_v(S, b, x, t_b, t_d)
            Vg *= (E2 | E2.T)[np.ix_(cb, cb)]
            if keep_lists:
                res.lists[g]["x"] = x
                res.lists[g]["E2"] = E2.copy()
        res.V[np.ix_(cols, cols)] += Vg
    return res

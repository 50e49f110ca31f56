"""Contracted Cartesian Gaussian basis functions (paper App. A, "Gaussian basis
functions": chi = sum_k c_k x^l y^m z^n exp(-a_k r^2) about the atom centre).

Reading (the paper gives only the primitive form): every Cartesian primitive
x^i y^j z^k exp(-a r^2) is normalised on its own,
    N = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2i-1)!! (2j-1)!! (2k-1)!!),
and the contraction is then rescaled to unit self-overlap.  For primitives of
the same centre and the same powers, normalised as above,
    <g_a | g_b> = (2 sqrt(ab) / (a + b))^(l + 3/2),
so the rescaling factor depends on the shell only.

Pins: unit self-overlap of every function (tests integrate chi^2 on a fine
radial x product grid and compare with 1), gradients against central
differences of the values, and the analytic overlap against numerical
quadrature.
"""
from __future__ import annotations

import math

import numpy as np

CART = {
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)],
}


def double_factorial(n: int) -> int:
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def primitive_norm(a: float, powers) -> float:
    i, j, k = powers
    l = i + j + k
    return ((2.0 * a / math.pi) ** 0.75 * (4.0 * a) ** (l / 2.0)
            / math.sqrt(double_factorial(2 * i - 1) * double_factorial(2 * j - 1)
                        * double_factorial(2 * k - 1)))


class Shell:
    """One shell: centre, angular momentum, exponents and the final
    per-component coefficients (raw coefficient x primitive norm x contraction
    rescale)."""

    def __init__(self, center, l, exps, raw_coefs):
        self.center = np.asarray(center, dtype=np.float64)
        self.l = int(l)
        self.exps = np.asarray(exps, dtype=np.float64)
        self.components = CART[self.l]
        a = self.exps
        c = np.asarray(raw_coefs, dtype=np.float64)
        # overlap of normalised primitives of equal powers
        ov = (2.0 * np.sqrt(np.outer(a, a)) / np.add.outer(a, a)) ** (self.l + 1.5)
        rescale = 1.0 / math.sqrt(float(c @ ov @ c))
        self.coefs = []  # one coefficient vector per Cartesian component
        for comp in self.components:
            n = np.array([primitive_norm(ai, comp) for ai in a])
            self.coefs.append(c * n * rescale)

    @property
    def size(self) -> int:
        return len(self.components)


def build_shells(xyz, basis) -> list:
    """Shells of a ``synth.Basis`` in basis-function order."""
    ptr = np.concatenate([[0], np.cumsum(basis.nprim)])
    return [Shell(xyz[basis.atom[s]], basis.l[s], basis.exps[ptr[s]:ptr[s + 1]],
                  basis.coefs[ptr[s]:ptr[s + 1]]) for s in range(len(basis.atom))]


def eval_basis(points: np.ndarray, shells: list, deriv: bool = False):
    """phi[i, mu] = chi_mu(r_i) (Eq. phi_def, transposed to points x functions);
    with ``deriv`` also dphi[c, i, mu] = d chi_mu / d r_c (c = x, y, z).

    chi = P(x, y, z) * g(r2),  P = x^i y^j z^k,  g = sum_k c_k exp(-a_k r2);
    d chi / dx = (dP/dx) g + P * sum_k c_k (-2 a_k x) exp(-a_k r2).
    """
    npts = points.shape[0]
    nbf = sum(s.size for s in shells)
    phi = np.zeros((npts, nbf))
    dphi = np.zeros((3, npts, nbf)) if deriv else None
    mu = 0
    for sh in shells:
        d = points - sh.center
        r2 = np.einsum("ij,ij->i", d, d)
        e = np.exp(-np.outer(r2, sh.exps))              # [npts, nprim]
        for comp, c in zip(sh.components, sh.coefs):
            g = e @ c
            poly = np.ones(npts)
            for ax in range(3):
                poly = poly * d[:, ax] ** comp[ax]
            phi[:, mu] = poly * g
            if deriv:
                gd = e @ (c * sh.exps)                   # sum c a exp(-a r2)
                for ax in range(3):
                    p = comp[ax]
                    dpoly = np.ones(npts) * p
                    for bx in range(3):
                        power = comp[bx] - (1 if bx == ax else 0)
                        if power < 0:
                            dpoly = np.zeros(npts)
                            break
                        dpoly = dpoly * d[:, bx] ** power
                    dphi[ax, :, mu] = dpoly * g - 2.0 * d[:, ax] * poly * gd
            mu += 1
    return phi, dphi


def overlap_matrix(shells: list) -> np.ndarray:
    """S_ij = int phi_i phi_j dr (Eq. overlap_matrix) by the Gaussian product
    theorem: each primitive pair is a Gaussian about P = (a A + b B)/(a + b)
    times exp(-ab/(a+b) |A-B|^2); the polynomial factors are expanded about P
    and integrated term by term, int t^n exp(-p t^2) dt = (n-1)!!/(2p)^(n/2)
    sqrt(pi/p) for even n.  Written independently of any other overlap code in
    the repository; used for the electron-count check."""
    funcs = []
    for sh in shells:
        for comp, c in zip(sh.components, sh.coefs):
            funcs.append((sh.center, comp, sh.exps, c))
    n = len(funcs)
    S = np.zeros((n, n))

    def one_dim(la, lb, xa, xb, xp, p):
        tot = 0.0
        for i in range(la + 1):
            for j in range(lb + 1):
                m = i + j
                if m % 2:
                    continue
                tot += (math.comb(la, i) * math.comb(lb, j) * (xp - xa) ** (la - i)
                        * (xp - xb) ** (lb - j)
                        * double_factorial(m - 1) / (2.0 * p) ** (m // 2) * math.sqrt(math.pi / p))
        return tot

    for i in range(n):
        A, pa_, ea, ca = funcs[i]
        for j in range(i, n):
            B, pb_, eb, cb = funcs[j]
            ab2 = float(np.sum((A - B) ** 2))
            tot = 0.0
            for a, c1 in zip(ea, ca):
                for b, c2 in zip(eb, cb):
                    p = a + b
                    P = (a * A + b * B) / p
                    v = math.exp(-a * b / p * ab2)
                    for ax in range(3):
                        v *= one_dim(pa_[ax], pb_[ax], A[ax], B[ax], P[ax], p)
                    tot += c1 * c2 * v
            S[i, j] = S[j, i] = tot
    return S

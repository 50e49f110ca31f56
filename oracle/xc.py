"""Exchange-correlation energy densities f(rho, sigma) (energy per volume) and
their derivatives v_rho = df/drho, v_sigma = df/dsigma, sigma = |grad rho|^2.

The paper states only that local and semilocal functionals are in scope
(Sec. III-F) and writes the potential v^xc_i of Eq. exc_quadrature; its own
experiments use M06-2X through Libxc, which is not reproducible here.  The
two functionals below are the ones the workloads name, spin-restricted:

  LDA exchange (Slater):  f = -(3/4) (3/pi)^(1/3) rho^(4/3)
  PBE-form GGA:            f = f_x + f_c
    exchange:     f_x = f_LDA * F(s),  F = 1 + kappa - kappa / (1 + mu s^2 / kappa),
                  s^2 = sigma / (4 (3 pi^2)^(2/3) rho^(8/3)),
                  kappa = 0.804, mu = beta pi^2 / 3
    correlation:  f_c = rho (eps_PW92(r_s) + H),  r_s = (3 / (4 pi rho))^(1/3),
                  eps_PW92 = -2 A (1 + a1 r_s) ln(1 + 1 / (2 A (b1 r_s^(1/2)
                             + b2 r_s + b3 r_s^(3/2) + b4 r_s^2))),
                  A = 0.031091, a1 = 0.21370, b1..b4 = 7.5957, 3.5876, 1.6382, 0.49294,
                  t^2 = sigma / (4 k_s^2 rho^2), k_s^2 = 4 k_F / pi, k_F = (3 pi^2 rho)^(1/3),
                  H = gamma ln(1 + (beta/gamma) t^2 (1 + B t^2) / (1 + B t^2 + B^2 t^4)),
                  B = (beta/gamma) / (exp(-eps_PW92 / gamma) - 1),
                  gamma = (1 - ln 2) / pi^2, beta = 0.06672455060314922.
  Points with rho < rho_min contribute nothing (f = v = 0).

Derivatives are taken by the complex step, v = Im f(x + i h) / h, which
differentiates exactly the expression above to rounding (no hand-derived
formula to get wrong).

Pins (tests): the Slater constant through the closed-form exchange energy of
a single s-Gaussian density; PBE exchange at sigma = 0 equals Slater; F(s)
limits 1 + mu s^2 and 1 + kappa; H -> beta t^2 for small t and eps + H -> 0
for large t; complex-step derivatives against central finite differences.
The PW92 fit constants through the published expansions of the uniform gas:
high density c0 = (1 - ln 2) / pi^2, c1 = 0.046644, no rs^(1/2) term,
c2 = 0.00664 (A, b1, b2, a1); low density d0 = 0.4335, d1 = 1.4408 (a1, b3,
b4).  The reduced gradients s^2, t^2 and beta, mu through the second-order
gradient coefficient of correlation (Ma-Brueckner, 0.004235 in Hartree units),
which PBE correlation reproduces and PBE exchange cancels at every density.
"""
from __future__ import annotations

import math

import numpy as np

RHO_MIN = 1e-14
CX = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)
KAPPA = 0.804
BETA = 0.06672455060314922
MU = BETA * math.pi ** 2 / 3.0
GAMMA = (1.0 - math.log(2.0)) / math.pi ** 2
PW_A, PW_A1 = 0.031091, 0.21370
PW_B = (7.5957, 3.5876, 1.6382, 0.49294)


def f_lda_x(rho):
    return -CX * rho ** (4.0 / 3.0)


def pbe_exchange_factor(s2):
    return 1.0 + KAPPA - KAPPA / (1.0 + MU * s2 / KAPPA)


def f_pbe_x(rho, sigma):
    s2 = sigma / (4.0 * (3.0 * math.pi ** 2) ** (2.0 / 3.0) * rho ** (8.0 / 3.0))
    return f_lda_x(rho) * pbe_exchange_factor(s2)


def eps_pw92(rs):
    b1, b2, b3, b4 = PW_B
    den = 2.0 * PW_A * (b1 * np.sqrt(rs) + b2 * rs + b3 * rs ** 1.5 + b4 * rs * rs)
    return -2.0 * PW_A * (1.0 + PW_A1 * rs) * np.log(1.0 + 1.0 / den)


def pbe_h(eps, t2):
    B = (BETA / GAMMA) / (np.exp(-eps / GAMMA) - 1.0)
    num = 1.0 + B * t2
    return GAMMA * np.log(1.0 + (BETA / GAMMA) * t2 * num / (num + B * B * t2 * t2))


def f_pbe_c(rho, sigma):
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    kf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    ks2 = 4.0 * kf / math.pi
    t2 = sigma / (4.0 * ks2 * rho * rho)
    eps = eps_pw92(rs)
    return rho * (eps + pbe_h(eps, t2))


def f_pbe(rho, sigma):
    return f_pbe_x(rho, sigma) + f_pbe_c(rho, sigma)


def evaluate(kind: str, rho: np.ndarray, sigma: np.ndarray | None, rho_min: float = RHO_MIN):
    """(f, v_rho, v_sigma) per point; v_sigma is zeros for LDA."""
    rho = np.asarray(rho, dtype=np.float64)
    f = np.zeros_like(rho)
    vr = np.zeros_like(rho)
    vs = np.zeros_like(rho)
    ok = rho >= rho_min
    r = rho[ok]
    h = 1e-20
    if kind == "lda_x":
        f[ok] = f_lda_x(r)
        vr[ok] = np.imag(f_lda_x(r + 1j * h * r)) / (h * r)
    elif kind == "pbe":
        s = np.maximum(np.asarray(sigma, dtype=np.float64)[ok], 0.0)
        f[ok] = f_pbe(r, s)
        vr[ok] = np.imag(f_pbe(r + 1j * h * r, s)) / (h * r)
        hs = h * np.maximum(s, r ** (8.0 / 3.0))
        vs[ok] = np.imag(f_pbe(r.astype(complex), s + 1j * hs)) / hs
    else:
        raise ValueError(kind)
    return f, vr, vs

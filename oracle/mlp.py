"""Learned per-point functional: a 2 -> 64 -> 64 -> 2 MLP surrogate of the
PBE-form GGA, its training loss, gradient and Adam update (FP64 reference).

TEST INFRASTRUCTURE: only tests, the smoke check and the benchmark's CPU
baseline use this module; the library never calls it.

The paper evaluates a semilocal functional per grid point between the two
block products (Sec. III-F, Eq. exc_quadrature: v_i feeds W = diag(w v)).  The
surrogate replaces that per-point evaluation.  Readings (the paper does not
describe a learned functional; these are the choices of this project):

  inputs   u1 = ln rho, u2 = ln max(sigma, SIGMA_FLOOR), mapped to
           z = (u - c) / s with the centre c and half-width s of the training
           box, so the box is [-1, 1]^2;
  network  h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), o = W3 h2 + b3
           (W1 64x2, W2 64x64, W3 2x64), FP16 weights, FP32 arithmetic on the
           GPU;
  outputs  o1 = F = f / e0(rho) (energy density over Slater exchange,
           e0 = -(3/4)(3/pi)^(1/3) rho^(4/3)), o2 = G = v_rho / v0(rho)
           (v0 = de0/drho = -(3/pi)^(1/3) rho^(1/3));
  v_sigma  the exact derivative of the network's energy density:
           v_sigma = e0 (d o1 / d z2) / (s2 sigma);
  fallback points outside the box use the analytic functional; points with
           rho < rho_min contribute nothing, as in the analytic path;
  loss     mean over valid points of (o1 - F*)^2 + (o2 - G*)^2 with targets
           F*, G* from the analytic PBE-form functional;
  update   Adam (Kingma & Ba 2015) with bias correction, FP32 master weights,
           FP16 copies for the forward pass.

Parameter vector (length NP = 4482, this order): W1 (64 x 2, row-major by
hidden unit), b1 (64), W2 (64 x 64, row = output unit), b2 (64), W3 (2 x 64),
b3 (2).

Pins (tests/test_oracle_mlp.py): the hand-written backward pass against
central finite differences of the loss; d o1 / d z2 and v_sigma against
finite differences of the network's energy density; the targets at sigma = 0
against Slater exchange plus PW92 correlation; the first Adam step equals
lr * sign(g) and Adam drives a quadratic to its minimum; degenerate weights
(W = 0) give the bias outputs and v_sigma = 0.
"""
from __future__ import annotations

import math

import numpy as np

from . import xc as oxc

NH = 64
SIGMA_FLOOR = 1e-30
# offsets into the parameter vector
O_W1 = 0
O_B1 = O_W1 + NH * 2
O_W2 = O_B1 + NH
O_B2 = O_W2 + NH * NH
O_W3 = O_B2 + NH
O_B3 = O_W3 + 2 * NH
NP = O_B3 + 2


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[O_W1:O_B1].reshape(NH, 2), p[O_B1:O_W2], p[O_W2:O_B2].reshape(NH, NH), p[O_B2:O_W3],
            p[O_W3:O_B3].reshape(2, NH), p[O_B3:NP])


def fp16_weights(p):
    """The forward pass uses the FP16 values of the FP32 master weights."""
    return np.asarray(p, dtype=np.float32).astype(np.float16).astype(np.float64)


class Box:
    """Training box in (ln rho, ln sigma): lo/hi per input."""

    def __init__(self, lo1, hi1, lo2, hi2):
        self.lo = np.array([lo1, hi1, lo2, hi2], dtype=np.float64)

    @property
    def centre(self):
        return np.array([(self.lo[0] + self.lo[1]) / 2, (self.lo[2] + self.lo[3]) / 2])

    @property
    def half(self):
        return np.array([(self.lo[1] - self.lo[0]) / 2, (self.lo[3] - self.lo[2]) / 2])

    def as_array(self):
        return self.lo.copy()


def slater(rho):
    """e0 = Slater exchange energy density and v0 = de0/drho."""
    e0 = -oxc.CX * rho ** (4.0 / 3.0)
    v0 = -(4.0 / 3.0) * oxc.CX * rho ** (1.0 / 3.0)
    return e0, v0


def inputs(rho, sigma, box):
    """z (n x 2) and whether each point lies in the box."""
    u = np.stack([np.log(rho), np.log(np.maximum(sigma, SIGMA_FLOOR))], axis=1)
    z = (u - box.centre[None, :]) / box.half[None, :]
    inside = np.all(np.abs(z) <= 1.0, axis=1)
    return z, inside


def forward(p, z):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1 = np.tanh(z @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ W3.T + b3
    return o, (h1, h2)


def do1_dz2(p, cache):
    """Derivative of o1 with respect to the second input, by the chain rule."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    h1, h2 = cache
    t1 = (1.0 - h1 * h1) * W1[:, 1][None, :]          # d h1 / d z2
    t2 = (1.0 - h2 * h2) * (t1 @ W2.T)                # d h2 / d z2
    return t2 @ W3[0]


def targets(rho, sigma):
    """F* = f / e0 and G* = v_rho / v0 of the analytic PBE-form functional."""
    f, vr, _ = oxc.evaluate("pbe", rho, sigma, rho_min=0.0)
    e0, v0 = slater(rho)
    return f / e0, vr / v0


def functional(p16, box, rho, sigma, rho_min=oxc.RHO_MIN):
    """(f, v_rho, v_sigma, used_network) per point for the surrogate with its
    analytic fallback outside the box."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    f = np.zeros_like(rho)
    vr = np.zeros_like(rho)
    vs = np.zeros_like(rho)
    ok = rho >= rho_min
    z = np.zeros((rho.size, 2))
    inside = np.zeros(rho.size, dtype=bool)
    z[ok], inside[ok] = inputs(rho[ok], sigma[ok], box)
    net = ok & inside
    if np.any(net):
        o, cache = forward(p16, z[net])
        d = do1_dz2(p16, cache)
        e0, v0 = slater(rho[net])
        f[net] = e0 * o[:, 0]
        vr[net] = v0 * o[:, 1]
        vs[net] = e0 * d / (box.half[1] * np.maximum(sigma[net], SIGMA_FLOOR))
    fb = ok & ~inside
    if np.any(fb):
        f[fb], vr[fb], vs[fb] = oxc.evaluate("pbe", rho[fb], sigma[fb], rho_min)
    return f, vr, vs, net


def loss_grad(p16, z, tF, tG, mask):
    """Mean squared error over the points with mask = 1 and its gradient with
    respect to the parameters, by a hand-written backward pass."""
    W1, b1, W2, b2, W3, b3 = unpack(p16)
    m = np.asarray(mask, dtype=np.float64)
    n = max(1.0, m.sum())
    o, (h1, h2) = forward(p16, z)
    r = o - np.stack([tF, tG], axis=1)
    loss = float(np.sum(m[:, None] * r * r) / n)
    do = 2.0 * m[:, None] * r / n                     # d loss / d o
    da2 = (do @ W3) * (1.0 - h2 * h2)                 # d loss / d (W2 h1 + b2)
    da1 = (da2 @ W2) * (1.0 - h1 * h1)                # d loss / d (W1 z + b1)
    g = np.zeros(NP)
    g[O_W1:O_B1] = (da1.T @ z).ravel()
    g[O_B1:O_W2] = da1.sum(axis=0)
    g[O_W2:O_B2] = (da2.T @ h1).ravel()
    g[O_B2:O_W3] = da2.sum(axis=0)
    g[O_W3:O_B3] = (do.T @ h2).ravel()
    g[O_B3:NP] = do.sum(axis=0)
    return loss, g


def adam(p, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def cosine_lr(step, total, lr0, lr1):
    """Learning rate of step `step` (0-based) of `total`: cosine from lr0 to lr1."""
    if total <= 1:
        return lr0
    return lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * step / (total - 1)))

"""Atom-centred integration grid, Becke partition, Morton order and 128-point
blocks (paper App. A, "Numerical integration grids"; App. B "Grid-Point Morton
Ordering", Eq. morton_code; Sec. III-B-2).

Readings where the paper is silent:
  * radial rule: Treutler-Ahlrichs M4 map r = (xi/ln 2) (1+x)^0.6 ln(2/(1-x))
    with xi = 1 on Chebyshev second-kind nodes x_i = cos(i pi/(n+1)),
    i = 1..n, whose weights for int_{-1}^{1} g(x) dx are
    pi/(n+1) sin(i pi/(n+1)); radial shells are listed by increasing r;
  * angular rule: a product rule, Gauss-Legendre in cos(theta) with n_theta
    nodes times 2 n_theta equally spaced azimuths phi_k = 2 pi k / (2 n_theta)
    (the Lebedev tables are not available);
  * pruning: the radial shells are split into equal index ranges, inner to
    outer, each with its own n_theta;
  * Becke partition with three iterations of p(mu) = 1.5 mu - 0.5 mu^3 and no
    atomic-size adjustment; weight = w_rad w_ang P_A(r) / sum_B P_B(r) over all
    atoms;
  * Morton key per Eq. morton_code on coordinates shifted by the minimum of
    the atom's own points, scaled by 128 per bohr, truncated and clamped to
    20 bits; points are grouped by atom (atom order), stably sorted by key
    within each atom; the concatenated list is cut into 128-point blocks and
    the last block is padded with copies of the last point at weight 0.

Pins: radial x angular quadrature of exp(-r^2) and of polynomials x^a y^b z^c
exp(-r^2) against closed forms; Becke weights sum to the plain atomic
weights (partition of unity); Morton key against a brute-force bit test.
"""
from __future__ import annotations

import functools
import math

import numpy as np


@functools.lru_cache(maxsize=None)
def treutler_radial(n: int, xi: float = 1.0, alpha: float = 0.6):
    i = np.arange(1, n + 1)
    theta = i * math.pi / (n + 1)
    x = np.cos(theta)
    wx = math.pi / (n + 1) * np.sin(theta)
    r = xi / math.log(2.0) * (1.0 + x) ** alpha * np.log(2.0 / (1.0 - x))
    dr = xi / math.log(2.0) * (alpha * (1.0 + x) ** (alpha - 1.0) * np.log(2.0 / (1.0 - x))
                               + (1.0 + x) ** alpha / (1.0 - x))
    w = wx * dr * r * r
    order = np.argsort(r)
    return r[order], w[order]


@functools.lru_cache(maxsize=None)
def angular_product(ntheta: int):
    """Unit vectors and weights (summing to 4 pi), theta-major order (cached:
    callers must not modify the returned arrays)."""
    t, wt = np.polynomial.legendre.leggauss(ntheta)
    nphi = 2 * ntheta
    phi = 2.0 * math.pi * np.arange(nphi) / nphi
    st = np.sqrt(1.0 - t * t)
    dirs = np.stack([np.outer(st, np.cos(phi)).ravel(),
                     np.outer(st, np.sin(phi)).ravel(),
                     np.repeat(t, nphi)], axis=1)
    w = np.repeat(wt, nphi) * (2.0 * math.pi / nphi)
    return dirs, w


def atom_points(center, nrad: int, ntheta_regions) -> tuple:
    """Points and radial x angular weights of one atom, generation order:
    radial shells by increasing r, then the angular points of that shell."""
    r, wr = treutler_radial(nrad)
    nreg = len(ntheta_regions)
    pts, wts = [], []
    for ir in range(nrad):
        region = min(ir * nreg // nrad, nreg - 1)
        dirs, wa = angular_product(ntheta_regions[region])
        pts.append(center + r[ir] * dirs)
        wts.append(wr[ir] * wa)
    return np.concatenate(pts), np.concatenate(wts)


def becke_s(mu: np.ndarray) -> np.ndarray:
    p = mu
    for _ in range(3):
        p = 1.5 * p - 0.5 * p ** 3
    return 0.5 * (1.0 - p)


def becke_weights(points: np.ndarray, owner: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """P_owner(r) / sum_B P_B(r), P_B(r) = prod_{C != B} s(mu_BC(r)),
    mu_BC = (|r - B| - |r - C|) / |B - C|, over all atoms."""
    natm = xyz.shape[0]
    if natm == 1:
        return np.ones(points.shape[0])
    dist = np.linalg.norm(points[:, None, :] - xyz[None, :, :], axis=2)   # [n, natm]
    Rab = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    P = np.ones_like(dist)
    for b in range(natm):
        others = np.arange(natm) != b
        mu = (dist[:, b:b + 1] - dist[:, others]) / Rab[b, others][None, :]
        P[:, b] = np.prod(becke_s(mu), axis=1)
    return P[np.arange(points.shape[0]), owner] / P.sum(axis=1)


def morton_code(q: np.ndarray) -> np.ndarray:
    """Eq. morton_code: m = sum_k z_k 2^(3k) + y_k 2^(3k+1) + x_k 2^(3k+2),
    k = 0..19, for integer lattice coordinates q[:, (x, y, z)]."""
    q = q.astype(np.int64)
    m = np.zeros(q.shape[0], dtype=np.int64)
    for k in range(20):
        m |= ((q[:, 2] >> k) & 1) << (3 * k)
        m |= ((q[:, 1] >> k) & 1) << (3 * k + 1)
        m |= ((q[:, 0] >> k) & 1) << (3 * k + 2)
    return m


def lattice(points: np.ndarray, scale: float = 128.0) -> np.ndarray:
    lo = points.min(axis=0)
    q = np.floor((points - lo) * scale).astype(np.int64)
    return np.clip(q, 0, (1 << 20) - 1)


class Grid:
    """points [N, 3], weights [N], atom_of [N], block size and counts; N is a
    multiple of the block size (padding points carry weight 0)."""

    def __init__(self, points, weights, atom_of, nreal, block, raw_w=None):
        self.points = points
        self.weights = weights
        self.atom_of = atom_of
        self.nreal = nreal
        self.block = block
        self.raw_w = raw_w

    @property
    def npoints(self) -> int:
        return self.points.shape[0]

    @property
    def nblocks(self) -> int:
        return self.npoints // self.block

    def fill_weights(self, xyz, blocks):
        """Becke-partitioned weights of the given blocks (the others stay as they are)."""
        B = self.block
        idx = np.concatenate([np.arange(b * B, (b + 1) * B) for b in blocks]) if len(blocks) else np.zeros(0, int)
        idx = idx[idx < self.nreal]
        chunk = 20000
        for i0 in range(0, idx.size, chunk):
            sel = idx[i0:i0 + chunk]
            self.weights[sel] = self.raw_w[sel] * becke_weights(self.points[sel], self.atom_of[sel], xyz)
        return self


def build_grid(Z, xyz, spec, weight_blocks=None) -> Grid:
    """The molecular grid.  ``weight_blocks`` (optional list of block indices)
    restricts the Becke partition to those blocks; other weights are NaN."""
    pts, raw_w, owner = [], [], []
    for a in range(len(Z)):
        p, w = atom_points(xyz[a], spec.nrad, spec.ntheta)
        order = np.argsort(morton_code(lattice(p)), kind="stable")
        pts.append(p[order])
        raw_w.append(w[order])
        owner.append(np.full(p.shape[0], a, dtype=np.int64))
    pts = np.concatenate(pts)
    raw_w = np.concatenate(raw_w)
    owner = np.concatenate(owner)
    nreal = pts.shape[0]
    B = spec.block
    npad = (-nreal) % B
    if npad:
        pts = np.concatenate([pts, np.repeat(pts[-1:], npad, axis=0)])
        raw_w = np.concatenate([raw_w, np.zeros(npad)])
        owner = np.concatenate([owner, np.repeat(owner[-1:], npad)])
    w = np.full(pts.shape[0], np.nan)
    w[nreal:] = 0.0
    g = Grid(pts, w, owner, nreal, B, raw_w)
    blocks = range(g.nblocks) if weight_blocks is None else weight_blocks
    return g.fill_weights(xyz, list(blocks))

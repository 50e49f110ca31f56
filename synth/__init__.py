"""Seeded synthetic inputs for the exchange-correlation quadrature workloads.

This module is the one place both sides draw their inputs from: the CPU oracle
(``oracle/``) and the GPU library (``paper_2605_10363_gb300``).  It produces only
what a caller of the method would hand to it -- atoms, a Cartesian Gaussian
basis specification, a density matrix D and the grid/threshold settings -- and
contains none of the method's arithmetic (no basis evaluation, no grid, no
screening, no functional).  The one piece of integral arithmetic here, the
analytic overlap matrix, exists only to orthonormalise the random occupied
orbitals that D is built from (D = 2 C C^T with C^T S C = I, the density-matrix
definition of the paper's Appendix A, "The density matrix", with the factor 2 of
a closed-shell occupation); the oracle carries its own, separately written
overlap for its electron-count check.

Units: bohr and Hartree.  All randomness is drawn from ``numpy.random.Generator``
(PCG64) seeded with the integers stated per workload.

Workloads (sizes follow the paper's synthetic stand-ins; the paper's molecules,
basis files and dataset are not available):

  1  two water-like units, O-H 0.96 A, 104.5 deg, O-O 3 A, random orientation
     (seed 1); s/p basis, 50 functions (seed 2); D from 10 orbitals (seed 3);
     30 radial x 128 angular points, unpruned; LDA exchange; t_b = t_d = 1e-12.
  2  33 waters at liquid density (0.0334 / A^3), O-O >= 2.6 A (seed 11);
     s/p/d basis with def2-SVP-like shell counts (825 functions); D localised
     per molecule (seed 12); 75 radial shells pruned by thirds to 50/128/288
     angular points; PBE-form GGA; t_b = t_d = 1e-10.
  3  1000 atoms (240 C, 80 N, 80 O, 600 H) in a sphere of 0.1 atoms/A^3,
     min distance 1.0 A (seed 21); 9000 functions; D localised per atom
     neighbourhood (seed 22); grid as workload 2.
  4  256 frames of 20..130 waters (sizes seed 31), each jittered 0.05 A rms
     (seed 32), own D (seed 33 + frame); grid as workload 2.
  5  167 waters (501 atoms, seed 41), D seed 43; grid as workload 2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ANGSTROM = 1.0 / 0.529177210903  # bohr per angstrom (CODATA 2018)

# Cartesian component order inside a shell: l=0: s; l=1: x y z;
# l=2: xx xy xz yy yz zz (the usual lexicographic order).
CART = {
    0: [(0, 0, 0)],
    1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
    2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)],
}

ELEMENT_ELECTRONS = {1: 1, 6: 6, 7: 7, 8: 8}


def ladder(k: int, amin: float = 0.1, amax: float = 50.0) -> float:
    """Even-tempered exponent ladder a_k = amin (amax/amin)^(k/11), k = 0..11."""
    return amin * (amax / amin) ** (k / 11.0)


# Shell recipes: (l, ladder indices) per element.  Workload 1: O 4s3p, H 3s1p
# (2*13 + 4*6 = 50 functions).  Workloads 2-5: heavy atoms 3s2p1d (15 Cartesian
# functions), H 2s1p (5 functions).
RECIPE_SP = {
    8: [(0, (9, 10, 11)), (0, (6, 7, 8)), (0, (3, 4, 5)), (0, (1, 2)),
        (1, (7, 8, 9)), (1, (4, 5, 6)), (1, (1, 2, 3))],
    1: [(0, (6, 7, 8)), (0, (3, 4, 5)), (0, (0, 1, 2)), (1, (2, 3))],
}
RECIPE_SVP = {
    6: [(0, (9, 10, 11)), (0, (5, 6, 7)), (0, (1, 2)), (1, (5, 6, 7)), (1, (1, 2, 3)), (2, (3, 4))],
    7: [(0, (9, 10, 11)), (0, (5, 6, 7)), (0, (1, 2)), (1, (5, 6, 7)), (1, (1, 2, 3)), (2, (3, 4))],
    8: [(0, (9, 10, 11)), (0, (5, 6, 7)), (0, (1, 2)), (1, (5, 6, 7)), (1, (1, 2, 3)), (2, (3, 4))],
    1: [(0, (5, 6, 7)), (0, (1, 2)), (1, (3, 4))],
}


@dataclass
class Basis:
    """Contracted Cartesian Gaussian shells.

    ``exps``/``coefs`` are the raw primitive exponents and contraction
    coefficients, concatenated shell after shell; ``prim_ptr[s]:prim_ptr[s+1]``
    indexes shell s.  Coefficients multiply *unnormalised* primitives
    x^i y^j z^k exp(-a r^2); normalisation is the method's business.
    """
    atom: np.ndarray      # int32 [nshell]
    l: np.ndarray         # int32 [nshell]
    nprim: np.ndarray     # int32 [nshell]
    exps: np.ndarray      # float64 [nprim_total]
    coefs: np.ndarray     # float64 [nprim_total]

    @property
    def nshell(self) -> int:
        return int(self.atom.size)

    @property
    def prim_ptr(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.nprim)]).astype(np.int64)

    @property
    def nbf(self) -> int:
        return int(sum(len(CART[int(l)]) for l in self.l))


@dataclass
class GridSpec:
    """Atom-centred grid settings: ``nrad`` radial shells; the radial shells are
    split into ``len(ntheta)`` equal index ranges (inner to outer) and range r
    uses an angular rule of ntheta[r] polar x 2*ntheta[r] azimuthal points."""
    nrad: int
    ntheta: tuple
    block: int = 128


@dataclass
class System:
    name: str
    Z: np.ndarray          # int32 [natm]
    xyz: np.ndarray        # float64 [natm, 3], bohr
    basis: Basis
    D: np.ndarray          # float64 [nbf, nbf], symmetric
    grid: GridSpec
    t_b: float
    t_d: float
    xc: str                # "lda_x" | "pbe"
    meta: dict = field(default_factory=dict)

    @property
    def nbf(self) -> int:
        return self.basis.nbf


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_frame() -> np.ndarray:
    """O at the origin, H-O-H angle 104.5 deg, O-H 0.96 A (bohr)."""
    r = 0.96 * ANGSTROM
    half = math.radians(104.5) / 2
    return np.array([[0.0, 0.0, 0.0],
                     [r * math.sin(half), 0.0, r * math.cos(half)],
                     [-r * math.sin(half), 0.0, r * math.cos(half)]])


def _spatial_order(points: np.ndarray) -> np.ndarray:
    """Order points along a coarse 3-D Z-curve (input atom order only)."""
    lo = points.min(axis=0)
    q = np.floor((points - lo) / (2.0 * ANGSTROM)).astype(np.int64)
    key = np.zeros(len(points), dtype=np.int64)
    for bit in range(10):
        for d in range(3):
            key |= ((q[:, d] >> bit) & 1) << (3 * bit + (2 - d))
    return np.argsort(key, kind="stable")


def water_cluster(nw: int, seed: int, density_per_A3: float = 0.0334,
                  min_oo_A: float = 2.6) -> tuple[np.ndarray, np.ndarray]:
    """nw water molecules, oxygens rejection-sampled in a sphere at the given
    number density with O-O >= min_oo, random orientations.  Molecules are
    listed along a coarse spatial curve (atom order O H H per molecule)."""
    rng = np.random.default_rng(seed)
    radius = (3.0 * nw / (4.0 * math.pi * density_per_A3)) ** (1.0 / 3.0) * ANGSTROM
    dmin = min_oo_A * ANGSTROM
    centers: list[np.ndarray] = []
    while len(centers) < nw:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        if centers and np.min(np.linalg.norm(np.asarray(centers) - p, axis=1)) < dmin:
            continue
        centers.append(p)
    centers_a = np.asarray(centers)
    order = _spatial_order(centers_a)
    frame = water_frame()
    xyz = []
    for i in order:
        R = random_rotation(rng)
        xyz.append(frame @ R.T + centers_a[i])
    Z = np.tile(np.array([8, 1, 1], dtype=np.int32), nw)
    return Z, np.concatenate(xyz, axis=0)


def two_waters(seed: int) -> tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    frame = water_frame()
    a = frame @ random_rotation(rng).T
    b = frame @ random_rotation(rng).T + np.array([3.0 * ANGSTROM, 0.0, 0.0])
    R = random_rotation(rng)
    xyz = np.concatenate([a, b]) @ R.T
    return np.array([8, 1, 1, 8, 1, 1], dtype=np.int32), xyz


def organic_cluster(seed: int, counts=((6, 240), (7, 80), (8, 80), (1, 600)),
                    density_per_A3: float = 0.1, min_dist_A: float = 1.0):
    rng = np.random.default_rng(seed)
    natm = sum(c for _, c in counts)
    radius = (3.0 * natm / (4.0 * math.pi * density_per_A3)) ** (1.0 / 3.0) * ANGSTROM
    dmin = min_dist_A * ANGSTROM
    pts: list[np.ndarray] = []
    while len(pts) < natm:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        if pts and np.min(np.linalg.norm(np.asarray(pts) - p, axis=1)) < dmin:
            continue
        pts.append(p)
    pts_a = np.asarray(pts)
    Z = np.concatenate([np.full(c, z, dtype=np.int32) for z, c in counts])
    Z = Z[rng.permutation(natm)]
    order = _spatial_order(pts_a)
    return Z[order], pts_a[order]


# ----------------------------------------------------------------------------
# basis
# ----------------------------------------------------------------------------

def make_basis(Z: np.ndarray, recipe: dict, seed: int, amin: float = 0.1) -> Basis:
    """Shells per the element recipe; contraction coefficients uniform in
    [0.3, 1], drawn once per element (seeded) so equal elements share a basis."""
    coef_table = {}
    for z in sorted(recipe):
        rng = np.random.default_rng([seed, int(z)])
        coef_table[z] = [rng.uniform(0.3, 1.0, size=len(ks)) for (_, ks) in recipe[z]]
    atom, ls, nprim, exps, coefs = [], [], [], [], []
    for a, z in enumerate(Z):
        for (l, ks), cs in zip(recipe[int(z)], coef_table[int(z)]):
            atom.append(a)
            ls.append(l)
            nprim.append(len(ks))
            exps.extend(ladder(k, amin) for k in ks)
            coefs.extend(cs.tolist())
    return Basis(np.asarray(atom, np.int32), np.asarray(ls, np.int32),
                 np.asarray(nprim, np.int32), np.asarray(exps, np.float64),
                 np.asarray(coefs, np.float64))


def basis_function_atoms(Z: np.ndarray, basis: Basis) -> np.ndarray:
    out = []
    for a, l in zip(basis.atom, basis.l):
        out.extend([int(a)] * len(CART[int(l)]))
    return np.asarray(out, np.int64)


# ----------------------------------------------------------------------------
# density matrix (input preparation only)
# ----------------------------------------------------------------------------

def _dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def _prim_norm(a: float, lx: int, ly: int, lz: int) -> float:
    l = lx + ly + lz
    return ((2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2.0)
            / math.sqrt(_dfact(2 * lx - 1) * _dfact(2 * ly - 1) * _dfact(2 * lz - 1)))


def _overlap_1d(la: int, lb: int, PA: np.ndarray, PB: np.ndarray, p: np.ndarray) -> np.ndarray:
    """int (x-A)^la (x-B)^lb exp(-p (x-P)^2) dx by binomial expansion about P."""
    out = np.zeros_like(p)
    for i in range(la + 1):
        for j in range(lb + 1):
            k = i + j
            if k % 2:
                continue
            m = _dfact(k - 1) / (2.0 * p) ** (k // 2) * np.sqrt(np.pi / p)
            out += math.comb(la, i) * math.comb(lb, j) * PA ** (la - i) * PB ** (lb - j) * m
    return out


def overlap_matrix(xyz: np.ndarray, basis: Basis) -> np.ndarray:
    """Analytic overlap S of the normalised contracted Cartesian functions."""
    ptr = basis.prim_ptr
    # flatten to primitive-level records per basis function
    fn_center, fn_pow, fn_pr = [], [], []
    for s in range(basis.nshell):
        a = basis.exps[ptr[s]:ptr[s + 1]]
        c = basis.coefs[ptr[s]:ptr[s + 1]]
        l = int(basis.l[s])
        for (lx, ly, lz) in CART[l]:
            d = c * np.array([_prim_norm(ai, lx, ly, lz) for ai in a])
            fn_center.append(xyz[basis.atom[s]])
            fn_pow.append((lx, ly, lz))
            fn_pr.append((a, d))
    nbf = len(fn_pow)
    # primitive table; the primitives of one function are contiguous
    pf, pa, pd = [], [], []
    for f, (a, d) in enumerate(fn_pr):
        for ai, di in zip(a, d):
            pf.append(f)
            pa.append(ai)
            pd.append(di)
    pf = np.asarray(pf)
    pa = np.asarray(pa)
    pd = np.asarray(pd)
    pc = np.asarray(fn_center)[pf]
    pw = np.asarray(fn_pow)[pf]
    fstart = np.searchsorted(pf, np.arange(nbf))
    S = np.zeros((nbf, nbf))
    npr = pf.size
    fchunk = max(1, 1_500_000 // (npr * 3))
    for f0 in range(0, nbf, fchunk):
        f1 = min(nbf, f0 + fchunk)
        i0 = fstart[f0]
        i1 = fstart[f1] if f1 < nbf else npr
        a = pa[i0:i1, None]
        b = pa[None, :]
        p = a + b
        A = pc[i0:i1, None, :]
        B = pc[None, :, :]
        AB2 = np.sum((A - B) ** 2, axis=-1)
        x = a * b / p * AB2
        # primitive pairs whose Gaussian-product factor exp(-x) is below 1e-30
        # contribute nothing at double precision and are left out
        r, c = np.nonzero(x < 69.0)
        ap, bp = pa[i0 + r], pa[c]
        pp = ap + bp
        v = np.exp(-x[r, c]) * pd[i0 + r] * pd[c]
        for dim in range(3):
            Ad, Bd = pc[i0 + r, dim], pc[c, dim]
            Pd = (ap * Ad + bp * Bd) / pp
            PA, PB = Pd - Ad, Pd - Bd
            la, lb = pw[i0 + r, dim], pw[c, dim]
            comp = np.empty_like(v)
            for li in range(3):
                for lj in range(3):
                    m = (la == li) & (lb == lj)
                    if m.any():
                        comp[m] = _overlap_1d(li, lj, PA[m], PB[m], pp[m])
            v = v * comp
        val = np.zeros(x.shape)
        val[r, c] = v
        cols = np.add.reduceat(val, fstart, axis=1)
        S[f0:f1] = np.add.reduceat(cols, fstart[f0:f1] - i0, axis=0)
    # renormalise contractions to unit self-overlap
    n = 1.0 / np.sqrt(np.diag(S))
    return S * n[:, None] * n[None, :]


def lowdin(C: np.ndarray, S: np.ndarray) -> np.ndarray:
    M = C.T @ S @ C
    w, U = np.linalg.eigh(M)
    return C @ (U * (1.0 / np.sqrt(w))) @ U.T


def density_random(nbf: int, nocc: int, S: np.ndarray, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    C = lowdin(rng.normal(size=(nbf, nocc)), S)
    return 2.0 * C @ C.T


def density_localised(supports: list, nbf: int, S: np.ndarray, seed: int) -> np.ndarray:
    """One orbital per support (list of basis indices), random normal
    coefficients on its support, then Loewdin-orthonormalised; D = 2 C C^T."""
    rng = np.random.default_rng(seed)
    C = np.zeros((nbf, len(supports)))
    for k, sup in enumerate(supports):
        C[sup, k] = rng.normal(size=len(sup))
    C = lowdin(C, S)
    D = 2.0 * C @ C.T
    return 0.5 * (D + D.T)


def density_variants(system: System, n: int, seed0: int = 100) -> list:
    """n further density matrices of a water-cluster system from its own recipe
    (one random orbital per occupied pair on each molecule, Loewdin-
    orthonormalised), seeds seed0 .. seed0 + n - 1: the densities an SCF or a
    trajectory passes through on the same geometry and grid."""
    S = overlap_matrix(system.xyz, system.basis)
    sups = _water_supports(system.Z, system.basis)
    return [density_localised(sups, system.nbf, S, seed0 + k) for k in range(n)]


def _water_supports(Z: np.ndarray, basis: Basis):
    fa = basis_function_atoms(Z, basis)
    sups = []
    for m in range(len(Z) // 3):
        idx = np.nonzero((fa >= 3 * m) & (fa < 3 * m + 3))[0]
        sups.extend([idx] * 5)  # 10 electrons -> 5 occupied orbitals
    return sups


def _atom_supports(Z: np.ndarray, xyz: np.ndarray, basis: Basis, radius_A: float = 1.6):
    fa = basis_function_atoms(Z, basis)
    sups = []
    electrons = 0
    for a, z in enumerate(Z):
        before = electrons
        electrons += ELEMENT_ELECTRONS[int(z)]
        norb = electrons // 2 - before // 2
        if norb == 0:
            continue
        near = np.nonzero(np.linalg.norm(xyz - xyz[a], axis=1) <= radius_A * ANGSTROM)[0]
        idx = np.nonzero(np.isin(fa, near))[0]
        sups.extend([idx] * norb)
    return sups


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

GRID_SMALL = GridSpec(nrad=30, ntheta=(8,))
GRID_PRUNED = GridSpec(nrad=75, ntheta=(5, 8, 12))


def make_system(config: int, frame: int = 0, nwaters: int | None = None, keep_overlap: bool = False) -> System:
    """The seeded synthetic system for one of the five workloads.

    ``nwaters`` overrides the cluster size (water workloads only) for small
    test variants of the same recipe.  ``keep_overlap`` keeps the overlap
    matrix built for D in ``meta["S"]``."""
    sysm = _make_system(config, frame, nwaters)
    if not keep_overlap:
        sysm.meta.pop("S", None)
    return sysm


def _make_system(config: int, frame: int, nwaters: int | None) -> System:
    if config == 1:
        Z, xyz = two_waters(1)
        basis = make_basis(Z, RECIPE_SP, 2)
        S = overlap_matrix(xyz, basis)
        D = density_random(basis.nbf, 10, S, 3)
        return System("two_waters_lda", Z, xyz, basis, D, GRID_SMALL, 1e-12, 1e-12, "lda_x", meta={"S": S})
    if config in (2, 5):
        nw = nwaters if nwaters is not None else (33 if config == 2 else 167)
        Z, xyz = water_cluster(nw, 11 if config == 2 else 41)
        basis = make_basis(Z, RECIPE_SVP, 2)
        S = overlap_matrix(xyz, basis)
        D = density_localised(_water_supports(Z, basis), basis.nbf, S, 12 if config == 2 else 43)
        name = f"water{nw}_pbe"
        return System(name, Z, xyz, basis, D, GRID_PRUNED, 1e-10, 1e-10, "pbe", meta={"S": S})
    if config == 3:
        Z, xyz = organic_cluster(21)
        basis = make_basis(Z, RECIPE_SVP, 2)
        S = overlap_matrix(xyz, basis)
        D = density_localised(_atom_supports(Z, xyz, basis), basis.nbf, S, 22)
        return System("cnoh1000_pbe", Z, xyz, basis, D, GRID_PRUNED, 1e-10, 1e-10, "pbe", meta={"S": S})
    if config == 4:
        sizes = np.random.default_rng(31).integers(20, 131, size=256)
        nw = int(sizes[frame]) if nwaters is None else nwaters
        Z, xyz = water_cluster(nw, 31_000 + nw)
        rng = np.random.default_rng([32, frame])
        xyz = xyz + rng.normal(scale=0.05 * ANGSTROM / math.sqrt(3.0), size=xyz.shape)
        basis = make_basis(Z, RECIPE_SVP, 2)
        S = overlap_matrix(xyz, basis)
        D = density_localised(_water_supports(Z, basis), basis.nbf, S, 33 + frame)
        return System(f"frame{frame}_water{nw}_pbe", Z, xyz, basis, D, GRID_PRUNED, 1e-10, 1e-10, "pbe",
                      meta={"frame": frame, "S": S})
    raise ValueError(f"unknown workload {config}")


def frame_sizes(nframes: int = 256) -> np.ndarray:
    """Water counts of the batched-frames workload (seed 31)."""
    return np.random.default_rng(31).integers(20, 131, size=256)[:nframes]


def shell_sizes(basis: Basis) -> np.ndarray:
    """Cartesian functions per shell."""
    return np.array([len(CART[int(l)]) for l in basis.l], dtype=np.int32)


def permute_shells(system: System, perm) -> System:
    """The same system with its shells in the order perm (position k holds old
    shell perm[k]); D is permuted to match.  Array bookkeeping only."""
    perm = np.asarray(perm, dtype=np.int64)
    b = system.basis
    pp = b.prim_ptr
    nfn = shell_sizes(b)
    foff = np.concatenate([[0], np.cumsum(nfn)]).astype(np.int64)
    prim_idx = np.concatenate([np.arange(pp[s], pp[s + 1]) for s in perm])
    fn_idx = np.concatenate([np.arange(foff[s], foff[s + 1]) for s in perm])
    nb = Basis(b.atom[perm].copy(), b.l[perm].copy(), b.nprim[perm].copy(), b.exps[prim_idx].copy(),
               b.coefs[prim_idx].copy())
    D = system.D[np.ix_(fn_idx, fn_idx)].copy()
    return System(system.name + "_reordered", system.Z, system.xyz, nb, D, system.grid, system.t_b, system.t_d,
                  system.xc, meta=dict(system.meta, shell_perm=perm, fn_perm=fn_idx))

# ---------------------------------------------------------------------------- learned functional inputs
MLP_HIDDEN = 64
MLP_NPARAMS = MLP_HIDDEN * 2 + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + 2 * MLP_HIDDEN + 2


def mlp_init(seed: int = 42) -> np.ndarray:
    """Seeded FP32 initial parameters of the 2 -> 64 -> 64 -> 2 surrogate
    (order W1, b1, W2, b2, W3, b3): Glorot-uniform weights, zero hidden biases,
    output biases (1, 1) (the network starts at Slater exchange)."""
    rng = np.random.default_rng(seed)
    h = MLP_HIDDEN

    def glorot(nout, nin):
        lim = math.sqrt(6.0 / (nin + nout))
        return rng.uniform(-lim, lim, size=(nout, nin))

    p = np.concatenate([glorot(h, 2).ravel(), np.zeros(h), glorot(h, h).ravel(), np.zeros(h),
                        glorot(2, h).ravel(), np.ones(2)])
    assert p.size == MLP_NPARAMS
    return p.astype(np.float32)


def mlp_box(rho: np.ndarray, sigma: np.ndarray, rho_lo: float = 1e-10, sigma_floor: float = 1e-30):
    """Training box (lo, hi of ln rho; lo, hi of ln sigma) of the points with
    rho >= rho_lo, as four doubles, widened by 1e-6 of each range so that the
    extreme points lie strictly inside."""
    rho = np.asarray(rho, dtype=np.float64)
    keep = rho >= rho_lo
    u1 = np.log(rho[keep])
    u2 = np.log(np.maximum(np.asarray(sigma, dtype=np.float64)[keep], sigma_floor))
    m1 = 1e-6 * (u1.max() - u1.min())
    m2 = 1e-6 * (u2.max() - u2.min())
    return np.array([u1.min() - m1, u1.max() + m1, u2.min() - m2, u2.max() + m2], dtype=np.float64)


def mlp_points(nsample: int, seed: int = 42) -> tuple[np.ndarray, np.ndarray]:
    """Seeded (rho, sigma) pairs spread over the ranges met on molecular grids
    (ln rho uniform in [ln 1e-10, ln 1e3], reduced gradient s in [0, 3]), for
    tests of the network that need no grid."""
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(math.log(1e-10), math.log(1e3), size=nsample))
    s = rng.uniform(0.0, 3.0, size=nsample)
    sigma = (s * 2.0 * (3.0 * math.pi ** 2) ** (1.0 / 3.0) * rho ** (4.0 / 3.0)) ** 2
    return rho, sigma

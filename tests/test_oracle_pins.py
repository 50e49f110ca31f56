"""Pins of the CPU oracle against facts fixed outside the oracle: closed forms,
exact invariants, textbook special cases, brute force and an independently
written second implementation (the input generator's overlap)."""
import math

import numpy as np
import pytest

import synth
from oracle import basis as ob
from oracle import exc as oe
from oracle import grid as og
from oracle import screen as osc
from oracle import xc as ox


def single_gaussian_system(a, kind="lda_x", nrad=100):
    Z = np.array([1])
    xyz = np.zeros((1, 3))
    bas = synth.Basis(np.array([0]), np.array([0]), np.array([1]), np.array([a]), np.array([1.0]))
    return synth.System("s", Z, xyz, bas, np.array([[2.0]]), synth.GridSpec(nrad, (8,)), 0.0, 0.0, kind)


# ---------------------------------------------------------------- closed form
@pytest.mark.parametrize("a,expected", [(0.5, -0.6819858182557268), (1.0, -0.9644735935233612),
                                        (2.0, -1.3639716365114531)])
def test_slater_exchange_single_s_gaussian(a, expected):
    """Restricted Slater exchange of a doubly occupied normalised s-Gaussian:
    E_x = -(3/4)(3/pi)^(1/3) 2^(4/3) (2a/pi)^2 (3 pi / 8a)^(3/2)."""
    s = single_gaussian_system(a)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    r = oe.evaluate(s, g, screened=False)
    assert abs(r.E - expected) < 1e-12
    assert abs(np.sum(g.weights * r.rho) - 2.0) < 1e-12


def test_density_and_gradient_of_single_s_gaussian():
    """A doubly occupied normalised s-Gaussian on the origin has
    rho = 2 (2a/pi)^(3/2) exp(-2 a r^2) and grad rho = -4 a r rho: the oracle's
    rho = Phi . (Phi D) and grad rho = 2 grad Phi . (Phi D) at the grid points."""
    a = 0.8
    s = single_gaussian_system(a, kind="pbe")
    g = og.build_grid(s.Z, s.xyz, s.grid)
    r = oe.evaluate(s, g, screened=False, want_v=False)
    p = g.points[:g.nreal]
    arg = 2.0 * a * np.sum(p * p, axis=1)
    rho = 2.0 * (2.0 * a / math.pi) ** 1.5 * np.exp(-arg)
    tol = 1e-14 + 1e-15 * arg               # exp's relative error grows with its argument
    assert np.all(np.abs(r.rho[:g.nreal] - rho) <= tol * rho)
    grad = -4.0 * a * p * rho[:, None]
    bound = 2.0 * (tol * rho)[:, None] * (4.0 * a * np.abs(p) + 1e-300)
    assert np.all(np.abs(r.grad[:g.nreal] - grad) <= bound)


# ---------------------------------------------------------------- grid
def test_radial_rule_gaussian_moments():
    r, w = og.treutler_radial(100)
    for n in (0, 2, 4):
        exact = math.gamma((n + 3) / 2) / 2.0  # int_0^inf r^(n+2) exp(-r^2) dr
        assert abs(np.sum(w * r ** n * np.exp(-r * r)) - exact) < 1e-12 * max(1, exact)


@pytest.mark.parametrize("nt", [5, 8, 12])
def test_angular_rule_polynomials(nt):
    dirs, w = og.angular_product(nt)
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    deg = nt - 1  # exact for all monomials up to this total degree (and beyond in theta)
    dfac = ob.double_factorial
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                val = np.sum(w * dirs[:, 0] ** a * dirs[:, 1] ** b * dirs[:, 2] ** c)
                if a % 2 or b % 2 or c % 2:
                    exact = 0.0
                else:
                    exact = 4 * math.pi * dfac(a - 1) * dfac(b - 1) * dfac(c - 1) / dfac(a + b + c + 1)
                assert abs(val - exact) < 1e-12, (a, b, c)


def test_becke_partition_of_unity():
    rng = np.random.default_rng(5)
    xyz = rng.normal(scale=2.0, size=(5, 3))
    pts = rng.normal(scale=3.0, size=(50, 3))
    tot = np.zeros(50)
    for a in range(5):
        tot += og.becke_weights(pts, np.full(50, a), xyz)
    assert np.allclose(tot, 1.0, atol=1e-14)


def test_becke_cell_function_closed_forms():
    """Becke's cell function (J. Chem. Phys. 88, 2547 (1988)): s = (1 - f_3) / 2,
    f_k the k-th iterate of p(mu) = 3 mu / 2 - mu^3 / 2.  Fixed values s(-1) = 1,
    s(0) = 1/2, s(1) = 0 and s(mu) + s(-mu) = 1.  Near mu = 1, p(1 - e) =
    1 - (3/2) e^2 (1 - e/3), so each iterate squares the distance from 1 and
    scales it by 3/2: 1 - f_3(1 - e) = (3/2)^7 e^8 (1 - 4e/3 + O(e^2)).  The e^8
    fixes three iterations (two give e^4, four e^16), the constant the
    polynomial's coefficients."""
    s = og.becke_s
    assert s(np.array(-1.0)) == 1.0 and s(np.array(0.0)) == 0.5 and s(np.array(1.0)) == 0.0
    mu = np.linspace(-1.0, 1.0, 41)
    assert np.abs(s(mu) + s(-mu) - 1.0).max() < 1e-15
    assert np.all(np.diff(s(mu)) < 0)
    for e in (0.05, 0.02):        # smaller e loses 1 - f_3 to cancellation in FP64
        r = s(np.array(1.0 - e)) / (0.5 * 1.5 ** 7 * e ** 8)
        assert abs(r - (1.0 - 4.0 * e / 3.0)) < 3.0 * e * e, (e, r)
    assert 200.0 < s(np.array(0.95)) / s(np.array(0.975)) < 300.0       # 2^8 (1 - 2e/3)


def test_becke_weights_at_nuclei_and_on_bisecting_planes():
    """At a nucleus the cell function of its own atom is 1 (mu = -1 against every
    other atom) and every other cell vanishes (its factor for this atom has
    mu = 1), so the own weight is exactly 1; on the plane bisecting two atoms of
    a diatomic both weights are exactly 1/2.  A sign error in mu puts the
    weight of a nucleus on the other atoms."""
    rng = np.random.default_rng(7)
    xyz = rng.normal(scale=2.0, size=(5, 3))
    for a in range(5):
        own = og.becke_weights(xyz[a:a + 1], np.array([a]), xyz)
        assert own[0] == 1.0
        for b in range(5):
            if b != a:
                assert og.becke_weights(xyz[a:a + 1], np.array([b]), xyz)[0] == 0.0
    two = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 2.0]])
    plane = np.array([[0.3, -0.7, 1.0], [1.5, 2.0, 1.0], [-4.0, 0.25, 1.0]])
    assert np.all(og.becke_weights(plane, np.zeros(3, int), two) == 0.5)
    near = np.array([[0.0, 0.0, 0.5], [0.2, 0.1, 0.3]])
    wa = og.becke_weights(near, np.zeros(2, int), two)
    wb = og.becke_weights(near, np.ones(2, int), two)
    assert np.all(wa > 0.9) and np.allclose(wa + wb, 1.0, atol=1e-15)


def test_morton_bits_brute_force():
    rng = np.random.default_rng(7)
    q = rng.integers(0, 1 << 20, size=(200, 3))
    m = og.morton_code(q)
    for i in range(200):
        for bit in range(60):
            k, which = divmod(bit, 3)
            coord = {0: 2, 1: 1, 2: 0}[which]   # bit 3k: z, 3k+1: y, 3k+2: x
            assert ((int(m[i]) >> bit) & 1) == ((int(q[i, coord]) >> k) & 1)


def test_grid_layout():
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    assert g.npoints % 128 == 0 and g.nreal == 6 * 30 * 128
    assert np.all(np.diff(g.atom_of[:g.nreal]) >= 0)
    for a in range(6):
        idx = np.nonzero(g.atom_of[:g.nreal] == a)[0]
        codes = og.morton_code(og.lattice(g.points[idx]))
        assert np.all(np.diff(codes) >= 0)
    # sum of Becke weights over all atoms' points reproduces a molecular integral:
    # the electron count check below covers it; here only positivity.
    assert np.all(g.weights[:g.nreal] >= 0)


# ---------------------------------------------------------------- basis
def test_basis_unit_norm_and_gradient():
    s = synth.make_system(1)
    shells = ob.build_shells(s.xyz, s.basis)
    one = [sh for sh in shells if np.allclose(sh.center, s.xyz[0])]
    pts, w = og.atom_points(s.xyz[0], 120, (16,))
    phi, dphi = ob.eval_basis(pts, one, deriv=True)
    norms = np.einsum("i,im->m", w, phi * phi)
    assert np.allclose(norms, 1.0, atol=1e-9)
    h = 1e-5
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fd = (ob.eval_basis(pts[:200] + e, one)[0] - ob.eval_basis(pts[:200] - e, one)[0]) / (2 * h)
        assert np.allclose(fd, dphi[ax, :200], atol=2e-6, rtol=1e-6)


def test_cartesian_component_order_and_norms():
    """Functions of a shell in the documented order s | x y z | xx xy xz yy yz
    zz: at a point r - A = (x, y, z) each d function is N_c x^i y^j z^k g(r), and
    for one primitive N_xx / N_xy = 1 / sqrt(3) ((2i-1)!! ratio), so
    chi_xy / chi_xx = sqrt(3) y / x and chi_xx / chi_yy = x^2 / y^2."""
    bas = synth.Basis(np.array([0, 0, 0]), np.array([0, 1, 2]), np.array([1, 1, 1]), np.array([0.7, 0.7, 0.7]),
                      np.array([1.0, 1.0, 1.0]))
    sh = ob.build_shells(np.zeros((1, 3)), bas)
    x, y, z = 0.3, -0.5, 0.8
    phi, _ = ob.eval_basis(np.array([[x, y, z]]), sh)
    s_, px, py, pz, dxx, dxy, dxz, dyy, dyz, dzz = phi[0]
    assert np.allclose([px / s_, py / s_, pz / s_], np.array([x, y, z]) * math.sqrt(4 * 0.7), rtol=1e-13)
    r3 = math.sqrt(3.0)
    assert np.allclose([dxy / dxx, dxz / dxx, dyz / dxx], [r3 * y / x, r3 * z / x, r3 * y * z / (x * x)], rtol=1e-13)
    assert np.allclose([dyy / dxx, dzz / dxx], [y * y / (x * x), z * z / (x * x)], rtol=1e-13)


def test_overlap_two_independent_implementations_and_quadrature():
    s = synth.make_system(1)
    shells = ob.build_shells(s.xyz, s.basis)
    S = ob.overlap_matrix(shells)
    S2 = synth.overlap_matrix(s.xyz, s.basis)
    assert np.abs(S - S2).max() < 1e-13
    g = og.build_grid(s.Z, s.xyz, synth.GridSpec(60, (14,)))
    phi, _ = ob.eval_basis(g.points, shells)
    Sq = phi.T @ (g.weights[:, None] * phi)
    assert np.abs(Sq - S).max() < 5e-5


# ---------------------------------------------------------------- functional
def test_xc_limits():
    rho = np.array([1e-3, 0.1, 1.0, 30.0])
    assert np.allclose(ox.f_pbe_x(rho, 0.0 * rho), ox.f_lda_x(rho), rtol=1e-15)
    s2 = np.array([1e-8, 1e8])
    F = ox.pbe_exchange_factor(s2)
    assert abs((F[0] - 1) / s2[0] - ox.MU) < 1e-6
    assert abs(F[1] - (1 + ox.KAPPA)) < 1e-7
    # PW92 high-density limit: d eps / d ln rs -> A
    r1, r2 = 1e-10, 1e-11
    slope = (ox.eps_pw92(r1) - ox.eps_pw92(r2)) / math.log(r1 / r2)
    assert abs(slope - ox.PW_A) < 1e-4
    eps = ox.eps_pw92(np.array([2.0]))
    assert abs(ox.pbe_h(eps, np.array([1e-9]))[0] / 1e-9 - ox.BETA) < 1e-6
    assert abs(eps[0] + ox.pbe_h(eps, np.array([1e12]))[0]) < 1e-6


def test_xc_derivatives_central_difference():
    rng = np.random.default_rng(3)
    rho = 10 ** rng.uniform(-5, 2, size=40)
    sigma = rho ** (8 / 3) * 10 ** rng.uniform(-3, 2, size=40)
    for kind in ("lda_x", "pbe"):
        f, vr, vs = ox.evaluate(kind, rho, sigma)
        fn = ox.f_lda_x if kind == "lda_x" else None
        h = 1e-6 * rho
        if kind == "lda_x":
            fd = (fn(rho + h) - fn(rho - h)) / (2 * h)
        else:
            fd = (ox.f_pbe(rho + h, sigma) - ox.f_pbe(rho - h, sigma)) / (2 * h)
            # v_sigma: exchange and correlation parts nearly cancel, so each part
            # is differenced on its own and the tolerance scales with the parts
            hs = 1e-4 * sigma
            fdx = (ox.f_pbe_x(rho, sigma + hs) - ox.f_pbe_x(rho, sigma - hs)) / (2 * hs)
            fdc = (ox.f_pbe_c(rho, sigma + hs) - ox.f_pbe_c(rho, sigma - hs)) / (2 * hs)
            assert np.all(np.abs(vs - (fdx + fdc)) <= 1e-6 * (np.abs(fdx) + np.abs(fdc)))
        assert np.allclose(vr, fd, rtol=1e-7)
    _, vr, _ = ox.evaluate("lda_x", rho, None)
    assert np.allclose(vr, -(3 / math.pi) ** (1 / 3) * rho ** (1 / 3), rtol=1e-14)


def test_rho_min_cut_is_strict():
    """Points with rho < rho_min contribute nothing; rho = rho_min itself counts."""
    rho = np.array([ox.RHO_MIN, ox.RHO_MIN * (1.0 - 1e-15), 0.0])
    for kind, sigma in (("lda_x", None), ("pbe", np.full(3, 1e-40))):
        f, vr, vs = ox.evaluate(kind, rho, sigma)
        assert f[0] < 0.0 and vr[0] < 0.0
        assert f[1] == 0.0 and vr[1] == 0.0 and vs[1] == 0.0 and f[2] == 0.0


# ---------------------------------------------------------------- quadrature invariants
@pytest.fixture(scope="module")
def w1():
    s = synth.make_system(1)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    return s, g, sh


def test_electron_count_and_symmetry(w1):
    s, g, sh = w1
    r = oe.evaluate(s, g, sh, screened=False)
    S = ob.overlap_matrix(sh)
    assert abs(np.sum(g.weights * r.rho) - np.trace(s.D @ S)) < 1e-3
    assert abs(np.trace(s.D @ S) - 20.0) < 1e-10
    assert np.array_equal(r.V, r.V.T)


def test_lda_trace_and_scaling(w1):
    s, g, sh = w1
    r = oe.evaluate(s, g, sh, screened=False)
    assert abs(np.sum(s.D * r.V) - 4.0 / 3.0 * r.E) < 1e-11 * abs(r.E)
    s2 = synth.System(s.name, s.Z, s.xyz, s.basis, 1.7 * s.D, s.grid, s.t_b, s.t_d, s.xc)
    r2 = oe.evaluate(s2, g, sh, screened=False, want_v=False)
    assert abs(r2.E - 1.7 ** (4 / 3) * r.E) < 1e-12 * abs(r.E)


def test_gga_trace_identity_and_derivative(w1):
    s, g, sh = w1
    r = oe.evaluate(s, g, sh, screened=False, xc_kind="pbe")
    sigma = np.sum(r.grad ** 2, axis=1)
    _, vr, vs = ox.evaluate("pbe", r.rho, sigma)
    rhs = np.sum(g.weights * (r.rho * vr + 2 * sigma * vs))
    assert abs(np.sum(s.D * r.V) - rhs) < 1e-11 * abs(rhs)
    # dE/dD_{mu nu} (symmetric perturbation) = V_{mu nu} + V_{nu mu}
    rng = np.random.default_rng(0)
    for _ in range(4):
        m, n = rng.integers(0, s.nbf, size=2)
        h = 1e-5
        dD = np.zeros_like(s.D)
        dD[m, n] += h
        dD[n, m] += h
        Ep = oe.evaluate(synth.System("", s.Z, s.xyz, s.basis, s.D + dD, s.grid, 0, 0, "pbe"), g, sh,
                         screened=False, want_v=False).E
        Em = oe.evaluate(synth.System("", s.Z, s.xyz, s.basis, s.D - dD, s.grid, 0, 0, "pbe"), g, sh,
                         screened=False, want_v=False).E
        fd = (Ep - Em) / (2 * h)
        an = r.V[m, n] + r.V[n, m] if m != n else r.V[m, m]
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (m, n, fd, an)


def test_dense_against_einsum_definition(w1):
    s, g, sh = w1
    pts = g.points[:128]
    w = g.weights[:128]
    phi, dphi = ob.eval_basis(pts, sh, deriv=True)
    rho = np.einsum("mn,im,in->i", s.D, phi, phi)
    grad = np.einsum("mn,cim,in->ic", s.D, dphi, phi) + np.einsum("mn,im,cin->ic", s.D, phi, dphi)
    sigma = np.sum(grad ** 2, axis=1)
    f, vr, vs = ox.evaluate("pbe", rho, sigma)
    V = (np.einsum("i,im,in->mn", w * vr, phi, phi)
         + 2 * np.einsum("i,ic,cim,in->mn", w * vs, grad, dphi, phi)
         + 2 * np.einsum("i,ic,im,cin->mn", w * vs, grad, phi, dphi))
    r = oe.evaluate(s, g, sh, screened=False, blocks=[0], xc_kind="pbe")
    assert np.allclose(r.rho[:128], rho, rtol=1e-13, atol=1e-16)
    assert np.allclose(r.grad[:128], grad, rtol=1e-12, atol=1e-15)
    assert abs(r.E - np.sum(w * f)) < 1e-14
    assert np.abs(r.V - V).max() < 1e-13


def test_screened_limits(w1):
    s, g, sh = w1
    blocks = [0, 40, 97, 179]
    dense = oe.evaluate(s, g, sh, screened=False, blocks=blocks, xc_kind="pbe")
    zero = oe.evaluate(s, g, sh, screened=True, blocks=blocks, xc_kind="pbe", t_b=0.0, t_d=0.0)
    assert np.array_equal(dense.rho, zero.rho) and np.array_equal(dense.V, zero.V)
    loose = oe.evaluate(s, g, sh, screened=True, blocks=blocks, xc_kind="pbe", t_b=1e-6, t_d=1e-6)
    # dropped pairs are bounded by t_d per element pair; the gap stays far below the bound
    assert abs(loose.E - dense.E) < 1e-4
    assert abs(loose.E - dense.E) > 0.0
    # V is a symmetric matrix by definition; screening drops whole block pairs
    # {p, q}, never one of the two mirror blocks (on these 20 grid blocks the
    # V rule's ordered pairs (p, q) and (q, p) differ)
    many = list(range(0, 180, 9))
    d20 = oe.evaluate(s, g, sh, screened=False, blocks=many, xc_kind="pbe")
    s20 = oe.evaluate(s, g, sh, screened=True, blocks=many, xc_kind="pbe", t_b=1e-6, t_d=1e-6)
    assert not np.array_equal(s20.V, d20.V)
    assert np.array_equal(s20.V, s20.V.T)


# ---------------------------------------------------------------- screening
def test_parallel_addressing_against_nonzero():
    rng = np.random.default_rng(11)
    for n in (1, 7, 32, 128, 1000):
        m = rng.random(n) < 0.3
        S, I = osc.parallel_addressing(m)
        assert S == m.sum() and np.array_equal(I, np.nonzero(m)[0])
    S, I = osc.parallel_addressing(np.zeros(64, bool))
    assert S == 0 and I.size == 0


def test_block_summaries_and_threshold_boundaries():
    """Block summaries are maxima of absolute values (Eq. block_summary_A), and
    the filters keep a block or pair whose value equals the threshold
    (Eq. block_filter_A: b_p >= t_b; Eq. block_pair_filter: a b >= t_d)."""
    D = np.zeros((64, 64))
    D[:32, :32] = -0.5
    D[3, 4] = 0.25
    D[40, 7] = -3.0
    dm = osc.d_block_max(D)
    assert np.array_equal(dm, [[0.5, 0.0], [3.0, 0.0]])
    M = np.zeros((128, 64))
    M[17, 40] = -2.0
    assert np.array_equal(osc.block_max_cols(M), [0.0, 2.0])
    t = 0.125
    assert np.array_equal(osc.retained(np.array([t, t / 2, 2 * t, 0.0]), t), [0, 2])
    b = np.array([0.5, 0.25])
    dmax = np.array([[0.5, 0.5], [0.5, 0.25]])
    E1 = osc.executed_rho(np.array([0, 1]), b, dmax, 0.25, 0.0625)      # b_p d b_q: 0.125, 0.0625, 0.015625
    assert E1.tolist() == [[True, True], [True, False]]
    x = np.array([0.5, 0.25])
    E2 = osc.executed_v(np.array([0, 1]), b, x, 0.25, 0.0625)           # b_p x_q: 0.25, 0.125, 0.125, 0.0625
    assert E2.all()


def test_executed_pairs_brute_force():
    rng = np.random.default_rng(2)
    nbf = 100
    D = rng.normal(size=(nbf, nbf)) * 10 ** rng.uniform(-14, 0, size=(nbf, nbf))
    D = D + D.T
    phi = rng.normal(size=(128, nbf)) * 10 ** rng.uniform(-14, 0, size=(1, nbf))
    t_b, t_d = 1e-9, 1e-8
    b = osc.block_max_cols(phi)
    S = osc.retained(b, t_b)
    dmax = osc.d_block_max(D)
    E1 = osc.executed_rho(S, b, dmax, t_b, t_d)
    nb = osc.nbasis_blocks(nbf)
    for p in range(nb):
        bp = max(abs(phi[i, mu]) for i in range(128) for mu in range(32 * p, min(nbf, 32 * p + 32)))
        assert (bp >= t_b) == (p in S)
    for i, p in enumerate(S):
        for j, q in enumerate(S):
            dm = max(abs(D[m, n]) for m in range(32 * p, min(nbf, 32 * p + 32))
                     for n in range(32 * q, min(nbf, 32 * q + 32)))
            assert E1[i, j] == (dm >= t_b and b[p] * dm * b[q] >= t_d)


# ---------------------------------------------------------------- PW92 / PBE constants
# Published coefficients of the spin-unpolarised uniform gas (Perdew & Wang,
# Phys. Rev. B 45, 13244 (1992)): high density eps_c = c0 ln rs - c1 + c2 rs ln rs
# - c3 rs + ..., with no rs^(1/2) term; low density eps_c = -d0 / rs + d1 / rs^(3/2) + ...
PW92_C1, PW92_C2 = 0.046644, 0.00664
PW92_D0, PW92_D1 = 0.4335, 1.4408
# Second-order gradient coefficient of correlation in the high-density limit
# (Ma & Brueckner; the Rasolt-Geldart form 0.001667 + 0.002568 at rs = 0),
# E_c^(2) = C_c int |grad rho|^2 / rho^(4/3), Hartree units.  PBE (Perdew, Burke,
# Ernzerhof, Phys. Rev. Lett. 77, 3865 (1996)) fixes beta so that H -> beta t^2
# reproduces it, and mu = beta pi^2 / 3 so that exchange cancels it.
MA_BRUECKNER_CC = 0.004235


def test_pw92_high_density_expansion():
    """The oracle's eps_PW92 fitted on rs in [1e-10, 1e-6]: log coefficient
    c0 = (1 - ln 2) / pi^2 (exact), constant -c1, no rs^(1/2) term, c2 rs ln rs.
    A typo in A, b1, b2 or a1 moves one of these."""
    rs = np.geomspace(1e-10, 1e-6, 40)
    M = np.stack([np.log(rs), np.ones_like(rs), np.sqrt(rs), rs * np.log(rs), rs], 1)
    c0, cst, half, c2, _ = np.linalg.lstsq(M, ox.eps_pw92(rs), rcond=None)[0]
    assert abs(c0 - (1.0 - math.log(2.0)) / math.pi ** 2) < 1e-6
    assert abs(-cst - PW92_C1) < 2e-6
    assert abs(half) < 2e-6
    assert abs(c2 - PW92_C2) < 1e-5


def test_pw92_low_density_expansion():
    """rs eps_PW92 fitted as a polynomial in u = rs^(-1/2) on rs in [1.1e3, 2.5e5]:
    intercept -d0 and slope d1 (pins a1 / b4 and a1 b3 / b4^2)."""
    u = np.linspace(0.002, 0.03, 40)
    c = np.polynomial.polynomial.polyfit(u, ox.eps_pw92(u ** -2) * u ** -2, 5)
    assert abs(-c[0] - PW92_D0) < 1e-4
    assert abs(c[1] - PW92_D1) < 5e-4


# PBE's published constants: the exchange enhancement is bounded by the local
# Lieb-Oxford bound, F_x <= 1.804 (kappa = 0.804), and beta = 0.066725.
PBE_FX_MAX = 1.804
PBE_BETA = 0.066725


def test_pbe_exchange_lieb_oxford_limit():
    """F_x(s) rises monotonically to the Lieb-Oxford value 1.804 as s grows."""
    s2 = np.geomspace(1e-6, 1e14, 60)
    F = ox.pbe_exchange_factor(s2)
    assert np.all(np.diff(F) > 0) and np.all(F < PBE_FX_MAX)
    assert abs(F[-1] - PBE_FX_MAX) < 1e-12


@pytest.mark.parametrize("s2", [0.25, 1.0, 4.0])
def test_pbe_correlation_high_density_scaling(s2):
    """Under uniform scaling to high density (r_s -> 0 at fixed s) PBE
    correlation per particle stays finite: H cancels the c0 ln r_s of eps_PW92
    because gamma = c0 = (1 - ln 2) / pi^2.  With t^2 = C s^2 / r_s,
    C = (pi / 4)(9 pi / 4)^(1/3), and B t^2 -> y = (beta / gamma) e^(-c1 / gamma) C s^2,
    the limit is -c1 + gamma ln((beta / gamma) C s^2 (1 + y) / (1 + y + y^2)),
    c1 = 0.046644 (PW92).  A wrong gamma makes the energy drift as ln r_s or
    vanish."""
    g = (1.0 - math.log(2.0)) / math.pi ** 2
    C = (math.pi / 4.0) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0)
    y = (PBE_BETA / g) * math.exp(-PW92_C1 / g) * C * s2
    limit = -PW92_C1 + g * math.log((PBE_BETA / g) * C * s2 * (1.0 + y) / (1.0 + y + y * y))
    for rs in (1e-6, 1e-8):
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        sigma = s2 * 4.0 * (3.0 * math.pi ** 2) ** (2.0 / 3.0) * rho ** (8.0 / 3.0)      # s^2 -> sigma
        eps = ox.f_pbe_c(np.array([rho]), np.array([sigma]))[0] / rho
        assert abs(eps - limit) < 2e-5, (rs, eps, limit)


@pytest.mark.parametrize("rho", [1e-4, 1e-2, 1.0, 1e2, 1e4])
def test_pbe_gradient_coefficients(rho):
    """d f / d sigma at sigma = 0 (complex step) times rho^(4/3): correlation
    gives the Ma-Brueckner coefficient at every density and exchange its
    negative.  A factor in s^2 or t^2 (k_F, k_s, the 4 or 2 of the reduced
    gradients), or a wrong beta or mu, moves them."""
    r = np.array([rho], dtype=complex)
    h = 1e-30 * rho ** (8.0 / 3.0)
    s = np.array([1j * h])
    cc = np.imag(ox.f_pbe_c(r, s))[0] / h * rho ** (4.0 / 3.0)
    cx = np.imag(ox.f_pbe_x(r, s))[0] / h * rho ** (4.0 / 3.0)
    assert abs(cc - MA_BRUECKNER_CC) < 1e-6
    assert abs(cx + MA_BRUECKNER_CC) < 1e-6

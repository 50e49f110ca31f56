"""The oracle's pins fail when a plausible mistake is planted in the oracle
(on the CPU, in memory, undone after each case): a wrong constant of the
PBE-form functional, a wrong iteration count or sign in the Becke partition,
a swapped Cartesian component order, block summaries without absolute values,
a strict instead of a non-strict threshold.  Each case names the pin that must
catch it; a pin that passes with the mistake in place is too weak."""
import math

import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import basis as ob
from oracle import grid as og
from oracle import screen as osc
from oracle import xc as ox


def _becke_s(iterations, a=1.5, b=0.5):
    def s(mu):
        p = mu
        for _ in range(iterations):
            p = a * p - b * p ** 3
        return 0.5 * (1.0 - p)
    return s


def _becke_weights_flipped(points, owner, xyz):
    dist = np.linalg.norm(points[:, None, :] - xyz[None, :, :], axis=2)
    R = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=2)
    P = np.ones_like(dist)
    for b in range(xyz.shape[0]):
        others = np.arange(xyz.shape[0]) != b
        P[:, b] = np.prod(og.becke_s((dist[:, others] - dist[:, b:b + 1]) / R[b, others][None, :]), axis=1)
    return P[np.arange(points.shape[0]), owner] / P.sum(axis=1)


def _d_block_max_signed(D, d=osc.D_BASIS):
    nb = osc.nbasis_blocks(D.shape[0], d)
    return np.array([[D[p * d:(p + 1) * d, q * d:(q + 1) * d].max() for q in range(nb)] for p in range(nb)])


_evaluate = ox.evaluate


def _evaluate_cutting_rho_min(kind, rho, sigma, rho_min=ox.RHO_MIN):
    f, vr, vs = _evaluate(kind, rho, sigma, rho_min)
    cut = np.asarray(rho) <= rho_min
    f[cut] = vr[cut] = vs[cut] = 0.0
    return f, vr, vs


CART_SWAPPED = dict(ob.CART)
CART_SWAPPED[2] = [(2, 0, 0), (1, 0, 1), (1, 1, 0), (0, 2, 0), (0, 1, 1), (0, 0, 2)]

CASES = [
    ("PBE kappa 0.800", ox, "KAPPA", 0.800, lambda: pins.test_pbe_exchange_lieb_oxford_limit()),
    ("PBE gamma (1 - ln 2) / pi", ox, "GAMMA", (1.0 - math.log(2.0)) / math.pi,
     lambda: pins.test_pbe_correlation_high_density_scaling(1.0)),
    ("PBE beta 0.0667", ox, "BETA", 0.0667, lambda: pins.test_pbe_gradient_coefficients(1.0)),
    ("PW92 A 0.0311", ox, "PW_A", 0.0311, lambda: pins.test_pw92_high_density_expansion()),
    ("PW92 b1 7.5", ox, "PW_B", (7.5, 3.5876, 1.6382, 0.49294), lambda: pins.test_pw92_high_density_expansion()),
    ("PW92 b4 0.48", ox, "PW_B", (7.5957, 3.5876, 1.6382, 0.48), lambda: pins.test_pw92_low_density_expansion()),
    ("Becke two iterations", og, "becke_s", _becke_s(2), lambda: pins.test_becke_cell_function_closed_forms()),
    ("Becke four iterations", og, "becke_s", _becke_s(4), lambda: pins.test_becke_cell_function_closed_forms()),
    ("Becke coefficients 1.49 / 0.49", og, "becke_s", _becke_s(3, 1.49, 0.49),
     lambda: pins.test_becke_cell_function_closed_forms()),
    ("Becke mu sign", og, "becke_weights", _becke_weights_flipped,
     lambda: pins.test_becke_weights_at_nuclei_and_on_bisecting_planes()),
    ("d order xy <-> xz", ob, "CART", CART_SWAPPED, lambda: pins.test_cartesian_component_order_and_norms()),
    ("D block maxima without abs", osc, "d_block_max", _d_block_max_signed,
     lambda: pins.test_block_summaries_and_threshold_boundaries()),
    ("retained with b > t_b", osc, "retained", lambda b, t: np.nonzero(b > t)[0],
     lambda: pins.test_block_summaries_and_threshold_boundaries()),
    ("rho_min itself cut", ox, "evaluate", _evaluate_cutting_rho_min, lambda: pins.test_rho_min_cut_is_strict()),
]


@pytest.mark.parametrize("name,module,attr,value,pin", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(monkeypatch, name, module, attr, value, pin):
    pin()                                          # passes on the oracle as written
    monkeypatch.setattr(module, attr, value)
    with pytest.raises(AssertionError):
        pin()

"""kldi_make_grid and kldi_screen refuse malformed input with a status and a
message before any device work (so these run without a GPU)."""
import numpy as np
import pytest

import synth


def _kldi():
    from paper_2605_10363_gb300 import kldi
    return kldi


@pytest.fixture(scope="module")
def water():
    kldi = _kldi()
    s = synth.make_system(2, nwaters=1)
    return s, kldi.make_grid(s.Z, s.xyz, s.grid.nrad, s.grid.ntheta)


def _screen(s, grid, xyz=None, atom=None, l=None, nprim=None, exps=None, coefs=None, t_b=None, prec="bf16x10",
            order=None):
    kldi = _kldi()
    b = s.basis
    pick = lambda v, d: d if v is None else v
    return kldi.screen(grid, s.Z, pick(xyz, s.xyz), pick(atom, b.atom), pick(l, b.l), pick(nprim, b.nprim),
                       pick(exps, b.exps), pick(coefs, b.coefs), pick(t_b, s.t_b), s.t_d, prec=prec, xc="pbe",
                       shell_order=order)


def _status(fn, *args, **kw):
    kldi = _kldi()
    with pytest.raises(kldi.KldiError) as e:
        fn(*args, **kw)
    return e.value.status, str(e.value)


def _with(a, i, v):
    a = np.array(a, copy=True)
    a[i] = v
    return a


def test_make_grid_refuses_non_finite_coordinates(water):
    kldi = _kldi()
    s, _ = water
    for bad in (np.nan, np.inf):
        st, msg = _status(kldi.make_grid, s.Z, _with(s.xyz, (1, 2), bad), s.grid.nrad, s.grid.ntheta)
        assert st == kldi.EINVAL and "atom 1" in msg
    assert _status(kldi.make_grid, s.Z, s.xyz, s.grid.nrad, [0])[0] == kldi.EINVAL
    assert _status(kldi.make_grid, s.Z, s.xyz, s.grid.nrad, s.grid.ntheta, block=64)[0] == kldi.EUNSUPPORTED


def test_screen_refuses_malformed_basis_and_molecule(water):
    kldi = _kldi()
    s, g = water
    b = s.basis
    cases = [
        (dict(exps=_with(b.exps, 3, -0.5)), kldi.EINVAL, "exponent"),
        (dict(exps=_with(b.exps, 0, 0.0)), kldi.EINVAL, "exponent"),
        (dict(exps=_with(b.exps, 2, np.inf)), kldi.EINVAL, "exponent"),
        (dict(coefs=_with(b.coefs, 1, np.nan)), kldi.EINVAL, "coefficient"),
        (dict(xyz=_with(s.xyz, (2, 0), np.nan)), kldi.EINVAL, "non-finite coordinate"),
        (dict(atom=_with(b.atom, 4, 3)), kldi.EINVAL, "atom=3"),
        (dict(atom=_with(b.atom, 0, -1)), kldi.EINVAL, "atom=-1"),
        (dict(nprim=_with(b.nprim, 0, 0)), kldi.EINVAL, "nprim=0"),
        (dict(l=_with(b.l, 0, 3)), kldi.EUNSUPPORTED, "l=3"),
        (dict(t_b=-1.0), kldi.EINVAL, "thresholds"),
        (dict(prec="tf32x3"), kldi.EUNSUPPORTED, "TF32X3"),
        (dict(order=np.zeros(len(b.l), np.int32)), kldi.EINVAL, "permutation"),
    ]
    for kw, want, text in cases:
        st, msg = _status(_screen, s, g, **kw)
        assert st == want and text in msg, (kw.keys(), st, msg)

"""kldi_grid_save / kldi_grid_load (host preprocessing, no GPU needed): a saved
grid loads back bit for bit, malformed files are refused with KLDI_EINVAL and
unreadable paths with KLDI_EIO, and kldi_screen refuses a grid whose owning
atoms are not in its molecule before it touches the device."""
import os
import struct

import numpy as np
import pytest

import synth

HEADER = 8 + 4 * 8


def _kldi():
    from paper_2605_10363_gb300 import kldi
    return kldi


@pytest.fixture(scope="module")
def saved(tmp_path_factory):
    kldi = _kldi()
    s = synth.make_system(2, nwaters=2)
    g = kldi.make_grid(s.Z, s.xyz, s.grid.nrad, s.grid.ntheta)
    path = str(tmp_path_factory.mktemp("grid") / "water2.grid")
    g.save(path)
    return s, g, path


def _raises(status, fn, *args):
    kldi = _kldi()
    with pytest.raises(kldi.KldiError) as e:
        fn(*args)
    assert e.value.status == status, e.value
    return e.value


def test_round_trip_is_bit_for_bit(saved):
    kldi = _kldi()
    _, g, path = saved
    h = kldi.load_grid(path)
    assert (h.npoints, h.nreal, h.nblocks) == (g.npoints, g.nreal, g.nblocks)
    assert g.nreal < g.npoints                     # the case has a padded last block
    for a, b in zip(g.export(), h.export()):
        assert a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))
    assert os.path.getsize(path) == HEADER + g.npoints * (4 * 8 + 4)
    with open(path, "rb") as f:
        assert f.read(8) == b"KLDIGRD1"
        assert struct.unpack("<4q", f.read(32)) == (g.npoints, g.nreal, g.nblocks, 128)


def _variant(tmp_path, path, name, edit):
    data = bytearray(open(path, "rb").read())
    edit(data)
    out = tmp_path / name
    out.write_bytes(bytes(data))
    return str(out)


def test_malformed_files_are_refused(saved, tmp_path):
    kldi = _kldi()
    _, g, path = saved
    n = g.npoints
    w_off = HEADER + 3 * 8 * n
    a_off = w_off + 8 * n

    def put(off, fmt, value):
        return lambda d: struct.pack_into(fmt, d, off, value)

    cases = {
        "magic": lambda d: d.__setitem__(slice(0, 1), b"X"),
        "truncated": lambda d: d.__delitem__(slice(len(d) - 4, len(d))),
        "longer": lambda d: d.extend(b"\0" * 8),
        "header_only": lambda d: d.__delitem__(slice(HEADER, len(d))),
        "short_header": lambda d: d.__delitem__(slice(20, len(d))),
        "nreal_zero_pad": put(8 + 8, "<q", g.npoints - 128),
        "nreal_too_big": put(8 + 8, "<q", g.npoints + 1),
        "block": put(8 + 24, "<q", 64),
        "nblocks": put(8 + 16, "<q", g.nblocks + 1),
        "negative_nblocks": put(8 + 16, "<q", -1),
        "padding_weight": put(w_off + 8 * (n - 1), "<d", 1e-3),
        "nan_weight": put(w_off, "<d", float("nan")),
        "inf_coordinate": put(HEADER + 8, "<d", float("inf")),
        "negative_atom": put(a_off + 4 * 5, "<i", -1),
    }
    for name, edit in cases.items():
        e = _raises(kldi.EINVAL, kldi.load_grid, _variant(tmp_path, path, name, edit))
        assert "kldi_grid_load" in str(e), name


def test_unreadable_and_unwritable_paths(saved, tmp_path):
    kldi = _kldi()
    _, g, _ = saved
    _raises(kldi.EIO, kldi.load_grid, str(tmp_path / "missing.grid"))
    _raises(kldi.EIO, g.save, str(tmp_path / "no_such_dir" / "x.grid"))
    assert not (tmp_path / "no_such_dir").exists()


def test_screen_refuses_a_grid_of_a_larger_molecule(saved):
    """The grid of two waters (6 atoms) with the basis and coordinates of one
    water (3 atoms): points owned by atoms 3-5 would index past the molecule's
    coordinates, so kldi_screen returns KLDI_EINVAL before any device work."""
    kldi = _kldi()
    _, g, path = saved
    one = synth.make_system(2, nwaters=1)
    for grid in (g, kldi.load_grid(path)):
        e = _raises(kldi.EINVAL, kldi.plan_for_system, one, "fp64", None, 0, 1e-14, None, grid)
        assert "atom" in str(e) and "3 atoms" in str(e)


@pytest.mark.gpu
def test_plan_from_a_loaded_grid_matches_a_fresh_one(saved):
    """kldi_exc on a plan built from the loaded grid gives the energy and V of
    the plan built from the grid it was saved from (FP64 block form; the V
    scatter's atomic order leaves differences at rounding level)."""
    kldi = _kldi()
    s, g, path = saved
    out = []
    for grid in (g, kldi.load_grid(path)):
        plan = kldi.plan_for_system(s, prec="fp64", xc="pbe", grid=grid)
        V = np.zeros((s.nbf, s.nbf))
        E = np.zeros(1)
        kldi.exc(plan, "pbe", s.D, V, E)
        out.append((E[0], V))
    (e0, v0), (e1, v1) = out
    assert abs(e1 - e0) <= 1e-13 * abs(e0)
    assert np.abs(v1 - v0).max() <= 1e-13 * np.abs(v0).max()
